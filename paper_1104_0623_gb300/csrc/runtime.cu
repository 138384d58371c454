// C ABI of the FIND library: handle, device workspace, per-level descriptor
// tables and the launch sequence of one solve.
//
// Execution of one pass over a batch of energies (on the caller's stream, the
// energies split into groups that run on up to 4 streams of the handle):
//   lead self-energies (closed form, unless given)
//   upward levels by height:   assemble -> LU of M(S,S) -> L by two triangular
//                              sweeps -> U (+T) (-> R)
//   downward levels by depth:  the same kernels on the complement clusters
//   leaf level:                assemble K -> invert K -> (G_K Sigma_K, .. G_K^H)
//                              -> extract diag G, diag G<, bond currents
// With FIND_FLAG_GRAPH the pass is captured once per call signature and
// replayed as a CUDA graph.  U and R of every cluster stay resident in one
// workspace allocation laid out [matrix id][energy][b][b]; per-level scratch,
// energy-major, holds M, Sigma_M, L, T and the pivots.
#include "../../include/find.h"
#include "kernels.cuh"
#include "plan.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using findgb::cplx;

namespace {

thread_local std::string g_create_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool device_accessible(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Byte arena used twice: once to size the descriptor tables, once to fill them.
struct Arena {
  std::vector<unsigned char> buf;
  template <class T>
  size_t put(const std::vector<T>& v) {
    size_t off = (buf.size() + 255) & ~size_t(255);
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

// Arithmetic of a GEMM or triangular-solve launch.
enum Arith { kFP64 = 0, kC64 = 1, kFF = 2 };

// One GEMM stage of a level: its ops and the tile maps of the six launch
// classes 2 * arith + big: [FP64 small, FP64 big, complex64 small, complex64
// big, float-float small, float-float big].
// The tensor-core products of a stage, in chunks whose digit planes fit the
// level's plane region (each chunk is one split and one product launch; the
// chunks of a stage run one after the other on the region).
struct TcChunk {
  findgb::TcLaunch L;
  size_t ops = 0, sitems = 0, ritems = 0, citems = 0, tmap = 0;  // arena offsets
  int nsitems = 0, nritems = 0, ncitems = 0, ntiles = 0;
  double fl = 0, by = 0;  // algorithmic flops and split bytes per energy
};

struct Stage {
  size_t ops = 0;
  size_t map[6] = {0, 0, 0, 0, 0, 0};  // arena offsets
  int nmap[6] = {0, 0, 0, 0, 0, 0};
  double fl[6] = {0, 0, 0, 0, 0, 0};   // algorithmic flops per energy of each class
  // the same with complex-symmetric outputs computed on their upper tiles
  // only (the mirrored launch): the flops those tiles execute
  double fl_sym[6] = {0, 0, 0, 0, 0, 0};
  std::vector<TcChunk> tc;
};

struct Level {
  bool leaf = false;
  int nops = 0, nrows = 0, max_s = 0;
  int rb = 16;                                 // triangular-solve row block
  int ntrsm[2] = {0, 0};                       // row blocks of [FP64, float-float] solves
  double by_asm = 0, by_ext = 0;               // per energy
  double fl_trsm[2] = {0, 0};
  size_t asmops = 0, row_op = 0, ext = 0, trsm = 0;  // arena offsets
  size_t trsm_map[2] = {0, 0};
  // LU (elimination levels) or inversion (leaf level) ops in four lists,
  // index df + 2 * in_smem: [FP64, float-float, FP64 in shared memory,
  // float-float in shared memory]
  // inversion / factorisation classes: bit 0 float-float, bit 1 shared-memory
  // inversion
  size_t inv[4] = {0, 0, 0, 0};
  int ninv[4] = {0, 0, 0, 0};
  int inv_max[4] = {0, 0, 0, 0};
  double fl_inv[4] = {0, 0, 0, 0};
  Stage st[3];
  int nstages = 0;
};

struct Layout {  // byte offsets inside the workspace
  size_t V, phi, eps, tau, E, sigL, sigR, modes, dles, U, R, scratch, oG, oGl, oJ, pos, bonds,
      status, meta, total;
};

// Tables of one handle laid out in the fixed device scratch (see
// find_solve_diag_static): the scratch address they were built for, the
// batch that fits, the layout, the levels and the host copy of the
// descriptor arena.
struct StaticView {
  unsigned char* base = nullptr;
  int ldl = -1;
  int batch = 0;
  Layout lay{};
  std::vector<Level> levels;
  std::vector<unsigned char> meta;
};

}  // namespace

struct find_handle {
  findgb::Plan plan;
  find_desc desc{};
  std::vector<double> V, phi, eps, tau;
  std::string err;
  // current workspace
  int batch = 0, lesser = -1;
  bool ldl = false;         // the current tables eliminate by LDL^T (else LU)
  bool ldl_build = false;   // the mode build_tables lays out
  // lesser tables that run every Sigma update (a caller's node-diagonal
  // Sigma< reaches every cluster), and the mode build_tables lays out
  bool sig_dense = false, sig_dense_build = false;
  unsigned char* ws = nullptr;
  Layout lay{};
  std::vector<Level> levels;  // upward, then downward, then the leaf level
  int n_up = 0, n_dn = 0;
  // profiling
  struct Pending { int cls; cudaEvent_t a, b; double flops, bytes; };
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  find_kernel_stat stats[19];
  // tables for the fixed device scratch
  StaticView sview;
  // streams and events of the concurrent energy groups of one pass
  std::vector<cudaStream_t> gstreams;
  std::vector<cudaEvent_t> gevents;
  // FIND_FLAG_GRAPH: captured passes, keyed by everything a pass's launches
  // bake in, replayed with cudaGraphLaunch; captured on cap_stream
  struct GraphKey {
    int nb, e0, lesser, bonds, sigL, sigR, dles, dles_per_e, sym;
    double fL, fR;
    bool operator==(const GraphKey& o) const {
      return nb == o.nb && e0 == o.e0 && lesser == o.lesser && bonds == o.bonds && sigL == o.sigL &&
             sigR == o.sigR && dles == o.dles && dles_per_e == o.dles_per_e && sym == o.sym &&
             fL == o.fL && fR == o.fR;
    }
  };
  struct Graph { GraphKey key; cudaGraphExec_t exec; };
  std::vector<Graph> graphs;  // most recently used last
  cudaStream_t cap_stream = nullptr;
  // the RGF baseline's own workspace (find_rgf_solve_lesser)
  unsigned char* rgf_ws = nullptr;
  int rgf_batch = 0;
  size_t rgf_meta_bytes = 0;
  size_t rgf_tab[3] = {0, 0, 0};  // GEMM ops, inversion ops, zero tile map (arena offsets)
};

namespace {

int fail(find_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return code;
}

int cuda_fail(find_handle* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? FIND_ENOMEM : FIND_ECUDA, m);
}

// Per-energy scratch of one elimination: M [, Sigma_M], L [, T], pivots; with
// the LDL^T elimination also W^T and W^T D^-1 (b x s each), D (2 s) and the
// block kinds (s ints after the pivots).
int64_t op_slot_elems(const findgb::ElimOp& op, bool lesser, bool ldl) {
  int64_t n = op.n, bs = (int64_t)op.b * op.s;
  int64_t piv = ((ldl ? 2 : 1) * (int64_t)op.s + 3) / 4;
  return (lesser ? 2 * n * n + 2 * bs : n * n + bs) + (ldl ? 2 * bs + 2 * (int64_t)op.s : 0) + piv;
}

int64_t leaf_slot_elems(const findgb::LeafOp& op, bool lesser) {
  int64_t n = op.n;
  return lesser ? 2 * n * n + 2 * (int64_t)op.c * n : n * n;
}

// Adds one GEMM op to a stage, assigning its tiles to the small or big class.
// Tile class of a product.  small_max > 0: 32x32 tiles when the larger output
// side is at most small_max.  small_max == 0 (default): 64x64 tiles unless
// their padded area exceeds the 32x32 tiling's by more than a margin: 20 %
// for float-float and complex64 (the big tile reloads and splits each operand
// half as often and measured ~20 % more efficient per useful flop), none for
// FP64 (both tiles keep the FP64 pipe nearly full, so padding decides).
bool big_tiles(int m, int n, int small_max, Arith arith) {
  if (small_max > 0) return std::max(m, n) > small_max;
  const double p64 = 4096.0 * ((m + 63) / 64) * ((n + 63) / 64);
  const double p32 = 1024.0 * ((m + 31) / 32) * ((n + 31) / 32);
  return p64 <= (arith == kFP64 ? 1.0 : 1.2) * p32;
}

void add_gemm(findgb::GemmOp g, std::vector<findgb::GemmOp>& ops, std::vector<int>* maps,
              Stage* st, Arith arith, int small_max) {
  if (g.m == 0 || g.n == 0) return;
  bool is_big = big_tiles(g.m, g.n, small_max, arith);
  const int cls = 2 * (int)arith + (is_big ? 1 : 0);
  const double kk = (double)(g.k + (g.A2 ? g.k2 : 0));
  st->fl[cls] += 8.0 * g.m * g.n * kk;
  int bm = is_big ? 64 : 32;
  int tm = (g.m + bm - 1) / bm, tn = (g.n + bm - 1) / bm;
  if (g.sym == 1) {
    for (int i = 0; i < tm; ++i)
      for (int j = i; j < tn; ++j)
        st->fl_sym[cls] += 8.0 * std::min(bm, g.m - i * bm) * std::min(bm, g.n - j * bm) * kk;
  } else {
    st->fl_sym[cls] += 8.0 * g.m * g.n * kk;
  }
  std::vector<int>& map = maps[cls];
  g.tile0 = (int)map.size();
  g.tiles_n = tn;
  int id = (int)ops.size();
  ops.push_back(g);
  for (int t = 0; t < tm * tn; ++t) map.push_back(id);
}

int rup(int x, int m) { return (x + m - 1) / m * m; }

// Digit planes of the tensor-core product that replaces GEMM g of arithmetic
// a, or 0 to keep g on the CUDA-core kernels: complex64 products stay there;
// so do products below tc_min in any dimension, products whose inner
// dimension exceeds the exact-accumulation limit of the planes (1024), and
// products whose padding to the 128 x 128 x 64 tiles wastes more than the
// tensor cores gain over the CUDA-core kernel of the same arithmetic
// (measured: about 12x over FP64, 5x over float-float).  Products that must
// match FP64 use the tensor cores only when tc_slices asks for it.
int tc_planes(const find_handle* h, const findgb::GemmOp& g, Arith a) {
  if ((h->desc.flags & FIND_FLAG_NO_TC) || a == kC64) return 0;
  const int k2 = g.A2 ? g.k2 : 0, kt = g.k + k2;
  const int mn = h->desc.tc_min > 0 ? h->desc.tc_min : 32;
  if (g.m < mn || g.n < mn || kt < mn || kt > 1024) return 0;
  const double used = (double)g.m * g.n * kt;
  const double padded = (double)rup(g.m, findgb::tc_tile_m()) * rup(g.n, findgb::tc_tile_n()) *
                        (rup(g.k, findgb::tc_tile_k()) + rup(k2, findgb::tc_tile_k()));
  if (used < (a == kFP64 ? 0.10 : 0.25) * padded) return 0;
  if (a == kFP64) return h->desc.tc_slices;  // 0: FP64 products stay on the CUDA cores
  return h->desc.tc_slices_mixed > 0 ? h->desc.tc_slices_mixed : 9;
}

findgb::TcOp tc_from_gemm(const findgb::GemmOp& g, int nsl) {
  findgb::TcOp t;
  std::memset(&t, 0, sizeof(t));
  t.m = g.m; t.n = g.n; t.k1 = g.k; t.k2 = g.A2 ? g.k2 : 0;
  // exactly accumulated diagonals: every one up to 5 (a diagonal of q + 1
  // pairs stays exact for (q + 1) K <= 8192, and the fixed-point sum of the
  // epilogue holds 6 of them); the rest share the last, rounded group
  t.nsl = nsl; t.nexact = std::min(nsl, 6);
  t.A1 = g.A; t.lda1 = g.lda; t.sa1 = g.sa; t.neg1 = g.alpha < 0.0;
  t.B1 = g.B; t.ldb1 = g.ldb; t.sb1 = g.sb; t.opb1 = g.opb;
  if (g.A2) {
    t.A2 = g.A2; t.lda2 = g.lda2; t.sa2 = g.sa2; t.neg2 = g.alpha2 < 0.0;
    t.B2 = g.B2; t.ldb2 = g.ldb2; t.sb2 = g.sb2; t.opb2 = g.opb2;
  }
  t.C = g.C; t.ldc = g.ldc; t.sc = g.sc; t.beta = g.beta;
  t.D = g.D; t.ldd = g.ldd; t.sd = g.sd;
  return t;
}

// Plane bytes per energy a chunk may take; a single larger op gets a chunk of
// its own.
constexpr int64_t kTcChunkBudget = int64_t(256) << 20;

// Groups the ops of a stage into chunks (the same for the same shapes, so the
// sizing and the real table builds agree).
std::vector<findgb::TcBuild> tc_chunks(const std::vector<findgb::TcOp>& ops) {
  std::vector<findgb::TcBuild> out;
  int64_t rows = 0, kp = 0, ints = 0;
  for (const auto& op : ops) {
    const int64_t r = 2LL * op.nsl * (rup(op.m, findgb::tc_tile_m()) + rup(op.n, findgb::tc_tile_n()));
    const int64_t k = rup(op.k1, findgb::tc_tile_k()) + rup(op.k2, findgb::tc_tile_k());
    const int64_t in = rup(op.m, findgb::tc_tile_m()) + rup(op.n, findgb::tc_tile_n());
    if (out.empty() || (rows > 0 && (rows + r) * std::max(kp, k) * 2 + 4 * (ints + in) > kTcChunkBudget)) {
      out.emplace_back();
      rows = 0; kp = 0; ints = 0;
    }
    rows += r; kp = std::max(kp, k); ints += in;
    findgb::tc_add_op(out.back(), op);
  }
  return out;
}

findgb::GemmOp gemm0() {
  findgb::GemmOp g;
  std::memset(&g, 0, sizeof(g));
  g.alpha = 1.0;
  g.alpha2 = 1.0;
  return g;
}

// Host-side bounds check of every operand a kernel will touch: each row-major
// block (rows x cols, leading dimension ld, per-energy stride) must lie inside
// [lo, hi) for all `batch` energies.  Run on the real tables before upload.
struct Bounds {
  const unsigned char* lo = nullptr;
  const unsigned char* hi = nullptr;
  // the level scratch: energy e owns [s_lo + e * s_stride, s_lo + (e+1) * s_stride)
  const unsigned char* s_lo = nullptr;
  const unsigned char* s_hi = nullptr;
  int64_t s_stride = 0;
  std::string err;
  void block(const cplx* p, int64_t rows, int64_t cols, int64_t ld, int64_t estride, int batch,
             const char* what) {
    if (!err.empty() || !lo || rows <= 0 || cols <= 0) return;
    if (!p || ld < cols) { err = std::string(what) + ": null pointer or ld < cols"; return; }
    const unsigned char* first = reinterpret_cast<const unsigned char*>(p);
    const unsigned char* last = reinterpret_cast<const unsigned char*>(
        p + (rows - 1) * ld + cols + (int64_t)(batch - 1) * estride);
    if (first < lo || last > hi) { err = std::string(what) + ": operand outside the workspace"; return; }
    if (s_lo && first >= s_lo && first < s_hi) {
      // a scratch operand: one energy's extent must stay inside that energy's
      // region, so concurrent energy groups never share scratch
      const int64_t off = (int64_t)(first - s_lo) % s_stride;
      const int64_t extent = ((rows - 1) * ld + cols) * (int64_t)sizeof(cplx);
      if ((int64_t)estride * (int64_t)sizeof(cplx) != s_stride || off + extent > s_stride)
        err = std::string(what) + ": scratch operand crosses its energy's region";
    }
  }
};

// Builds every level's descriptor tables into `ar`, with device pointers
// computed from `base` (the workspace address; 0 for sizing).
void build_tables(find_handle* h, unsigned char* base, const Layout& L, int batch, bool lesser,
                  Arena& ar_out, std::vector<Level>& levels_out, int64_t& scratch_elems,
                  Bounds* bc = nullptr, int* map_err = nullptr) {
  const findgb::Plan& p = h->plan;
  cplx* U = reinterpret_cast<cplx*>(base + L.U);
  cplx* R = lesser ? reinterpret_cast<cplx*>(base + L.R) : nullptr;
  cplx* S0 = reinterpret_cast<cplx*>(base + L.scratch);
  auto umat = [&](int id) { return id < 0 ? (cplx*)nullptr : U + p.mat_off[id] * batch; };
  auto rmat = [&](int id) { return (id < 0 || !R) ? (cplx*)nullptr : R + p.mat_off[id] * batch; };
  // Sigma< sparsity (Sec. 4.3): Sigma< is nonzero only on the contact columns
  // y = 0 and y = Ny - 1 (and on a caller's node-diagonal term), so a cluster
  // with no contact node has Sigma_M = 0 in its upward merge, and every term
  // of Eq. (7) vanishes: R = 0.  Its T and R products are skipped, R is never
  // stored, and the merges that read it take zeros.
  std::vector<char> zsig(p.mat_dim.size(), 0);
  if (lesser && !h->sig_dense_build)
    for (size_t c = 0; c < p.cl.size(); ++c) {
      const int id = p.up_mat[c];
      if (id >= 0 && p.cl[c].y0 > 0 && p.cl[c].y1 < p.ny) zsig[id] = 1;
    }
  auto rsrc = [&](int id) { return (id >= 0 && zsig[id]) ? (cplx*)nullptr : rmat(id); };
  scratch_elems = 0;
  // the LDL^T elimination (FP64 path, A = A^T) or the LU one
  const bool ldl = h->ldl_build;
  const bool mixed = h->desc.precision == FIND_MIXED || h->desc.precision == FIND_MIXED_FF;
  const bool ff_all = h->desc.precision == FIND_MIXED_FF;
  // shared-memory inversion only on request: measured slower than the
  // global-memory kernel (one 200 KB CTA per SM cannot hide its barriers)
  const int small_max = h->desc.gemm_small_max;  // 0: chosen per product by padding
  const int inv_smem = h->desc.invert_smem <= 0 ? 0
                       : std::min(h->desc.invert_smem, findgb::invert_smem_max());
  const int top_levels = h->desc.fp64_top_levels < 0 ? 2 : h->desc.fp64_top_levels;
  auto gemm_ok = [&](const findgb::GemmOp& q) {
    if (!bc || q.m == 0 || q.n == 0) return;
    // the kernels apply alpha as a sign
    if ((q.alpha != 1.0 && q.alpha != -1.0) || (q.A2 && q.alpha2 != 1.0 && q.alpha2 != -1.0))
      if (bc->err.empty()) bc->err = "gemm alpha must be +1 or -1";
    bc->block(q.A, q.m, q.k, q.lda, q.sa, batch, "gemm A");
    if (q.opb == 0) bc->block(q.B, q.k, q.n, q.ldb, q.sb, batch, "gemm B");
    else bc->block(q.B, q.n, q.k, q.ldb, q.sb, batch, "gemm B^H");
    if (q.A2) {
      bc->block(q.A2, q.m, q.k2, q.lda2, q.sa2, batch, "gemm A2");
      if (q.opb2 == 0) bc->block(q.B2, q.k2, q.n, q.ldb2, q.sb2, batch, "gemm B2");
      else bc->block(q.B2, q.n, q.k2, q.ldb2, q.sb2, batch, "gemm B2^H");
    }
    if (q.C) bc->block(q.C, q.m, q.n, q.ldc, q.sc, batch, "gemm C");
    bc->block(q.D, q.m, q.n, q.ldd, q.sd, batch, "gemm D");
  };

  // Scratch is energy-major: energy e owns [e * escr, (e + 1) * escr) for
  // every level, and a level lays its ops out inside that region.  Energy
  // groups running concurrently on different streams (at different levels)
  // therefore never touch each other's scratch.
  int64_t escr = 0;
  for (const auto& lvops : p.up_levels) {
    int64_t t = 0;
    for (const auto& op : lvops) t += op_slot_elems(op, lesser, ldl);
    escr = std::max(escr, t);
  }
  for (const auto& lvops : p.dn_levels) {
    int64_t t = 0;
    for (const auto& op : lvops) t += op_slot_elems(op, lesser, ldl);
    escr = std::max(escr, t);
  }
  {
    int64_t t = 0;
    for (const auto& op : p.leaf_ops) t += leaf_slot_elems(op, lesser);
    escr = std::max(escr, t);
  }
  escr = (escr + 15) & ~int64_t(15);  // keep every energy's region 256-byte aligned

  // The digit planes of a level's tensor-core products live in each energy's
  // scratch region after the level's op slots; escr is sized by a dry build.
  auto finish_tc = [&](Level& lv, std::vector<findgb::TcOp>* tcq, int nst, int64_t slot_end, Arena& arx,
                       bool dry, int64_t& need) {
    const int64_t off = (slot_end + 63) & ~int64_t(63);  // 1 KiB aligned within the region
    unsigned char* region = reinterpret_cast<unsigned char*>(S0 + off);
    for (int k = 0; k < nst; ++k) {
      for (auto& b : tc_chunks(tcq[k])) {
        int64_t oA = 0, oB = 0, oS = 0;
        const int64_t bytes = findgb::tc_slab_bytes(b, &oA, &oB, &oS);
        need = std::max(need, off + (bytes + 15) / 16);
        if (dry) continue;
        TcChunk c;
        c.L.slab.a = reinterpret_cast<unsigned short*>(region + oA);
        c.L.slab.b = reinterpret_cast<unsigned short*>(region + oB);
        c.L.slab.pitch = b.pitch;
        c.L.slab.plane_estride = escr * (int64_t)(sizeof(cplx) / 2);
        c.L.slab.scale = reinterpret_cast<int*>(region + oS);
        c.L.slab.scale_estride = escr * (int64_t)(sizeof(cplx) / 4);
        c.L.scale_ints = b.scale_ints;
        if (bc && bc->err.empty()) {
          if ((off * 16 + bytes) > escr * 16) bc->err = "tensor-core planes outside the energy's scratch";
          for (const auto& t : b.ops) {
            bc->block(t.A1, t.m, t.k1, t.lda1, t.sa1, batch, "tc A1");
            if (t.opb1 == 0) bc->block(t.B1, t.k1, t.n, t.ldb1, t.sb1, batch, "tc B1");
            else bc->block(t.B1, t.n, t.k1, t.ldb1, t.sb1, batch, "tc B1^H");
            if (t.A2) {
              bc->block(t.A2, t.m, t.k2, t.lda2, t.sa2, batch, "tc A2");
              if (t.opb2 == 0) bc->block(t.B2, t.k2, t.n, t.ldb2, t.sb2, batch, "tc B2");
              else bc->block(t.B2, t.n, t.k2, t.ldb2, t.sb2, batch, "tc B2^H");
            }
            if (t.C) bc->block(t.C, t.m, t.n, t.ldc, t.sc, batch, "tc C");
            bc->block(t.D, t.m, t.n, t.ldd, t.sd, batch, "tc D");
            if (t.nexact > 6 || t.k1 + t.k2 > 1024) bc->err = "tc op outside the exact range";
          }
        }
        if (map_err && base) {
          if (findgb::tc_encode_map(c.L.mapA, c.L.slab.a, b.pitch, b.rowsA, batch, escr * 16) ||
              findgb::tc_encode_map(c.L.mapB, c.L.slab.b, b.pitch, b.rowsB, batch, escr * 16))
            *map_err = 1;
        }
        for (const auto& t : b.ops) {
          const double kt = t.k1 + t.k2;
          c.fl += 8.0 * t.m * t.n * kt;
          c.by += 16.0 * (t.m + t.n) * kt +
                  2.0 * 2 * t.nsl * ((double)t.mt * 128 + (double)t.tiles_n * 128) * t.kp;
        }
        c.ops = arx.put(b.ops);
        c.sitems = arx.put(b.scale_items);
        c.ritems = arx.put(b.row_items);
        c.citems = arx.put(b.col_items);
        c.tmap = arx.put(b.tile_op);
        c.nsitems = (int)b.scale_items.size();
        c.nritems = (int)b.row_items.size();
        c.ncitems = (int)b.col_items.size();
        c.ntiles = (int)b.tile_op.size();
        lv.st[k].tc.push_back(c);
      }
    }
  };

  auto elim_level = [&](const std::vector<findgb::ElimOp>& ops, Arena& arx, std::vector<Level>& lvx,
                        bool dry, int64_t& need) {
    Level lv;
    std::vector<findgb::AsmOp> asmops;
    std::vector<int> row_op;
    std::vector<findgb::InvOp> inv[4];
    std::vector<findgb::TrsmOp> trs;
    std::vector<int> trs_map[2];
    std::vector<findgb::GemmOp> g[2];
    std::vector<int> maps[2][6];
    std::vector<findgb::TcOp> tcq[2];
    auto route = [&](const findgb::GemmOp& q, int k, Arith a) {
      const int nsl = tc_planes(h, q, a);
      if (nsl > 0 && q.m > 0 && q.n > 0) tcq[k].push_back(tc_from_gemm(q, nsl));
      else add_gemm(q, g[k], maps[k], &lv.st[k], a, small_max);
    };
    for (const auto& op : ops) lv.max_s = std::max(lv.max_s, op.s);
    lv.rb = findgb::trsm_rows_per_block(lv.max_s);
    int64_t off = 0;
    for (const auto& op : ops) {
      const int64_t slot = op_slot_elems(op, lesser, ldl);
      cplx* M = S0 + off;  // energy e at M + e * escr
      cplx* Sg = M + (int64_t)op.n * op.n;
      cplx* Lm = M + (lesser ? 2 : 1) * (int64_t)op.n * op.n;
      cplx* T = Lm + (int64_t)op.b * op.s;
      cplx* Wt = Lm + (lesser ? 2 : 1) * (int64_t)op.b * op.s;  // LDL^T only
      cplx* Yd = Wt + (int64_t)op.b * op.s;
      cplx* dv = Yd + (int64_t)op.b * op.s;
      int* piv = reinterpret_cast<int*>(ldl ? dv + 2 * (int64_t)op.s
                                            : Lm + (lesser ? 2 : 1) * (int64_t)op.b * op.s);
      off += slot;
      const int n = op.n, s = op.s, b = op.b;
      findgb::AsmOp a;
      a.n = n;
      a.row0 = lv.nrows;
      a.pos = op.pos;
      a.u1 = umat(op.src1); a.r1 = rsrc(op.src1); a.d1 = op.src1 < 0 ? 0 : p.mat_dim[op.src1];
      a.u2 = umat(op.src2); a.r2 = rsrc(op.src2); a.d2 = op.src2 < 0 ? 0 : p.mat_dim[op.src2];
      a.M = M;
      a.estride = escr;
      const bool sig_op = lesser && !(op.dst >= 0 && zsig[op.dst]);
      a.sig = sig_op ? 1 : 0;
      for (int r = 0; r < n; ++r) row_op.push_back((int)asmops.size());
      lv.nrows += n;
      asmops.push_back(a);
      if (bc) {
        bc->block(M, lesser ? 2 * (int64_t)n : n, n, n, escr, batch, "assemble M");
        if (a.u1) bc->block(a.u1, a.d1, a.d1, a.d1, (int64_t)a.d1 * a.d1, batch, "source U1");
        if (a.u2) bc->block(a.u2, a.d2, a.d2, a.d2, (int64_t)a.d2 * a.d2, batch, "source U2");
        if (a.r1) bc->block(a.r1, a.d1, a.d1, a.d1, (int64_t)a.d1 * a.d1, batch, "source R1");
        if (a.r2) bc->block(a.r2, a.d2, a.d2, a.d2, (int64_t)a.d2 * a.d2, batch, "source R2");
        const int pw = ((ldl ? 2 : 1) * s + 3) / 4;
        if (s > 0) bc->block(reinterpret_cast<const cplx*>(piv), 1, pw, pw, escr, batch, "pivots");
        for (int q = 0; q < n && bc->err.empty(); ++q) {
          const findgb::Pos& pq = p.pos[op.pos + q];
          int d = pq.src == 1 ? a.d1 : pq.src == 2 ? a.d2 : 1;
          if (pq.idx < 0 || pq.idx >= d || pq.node < 0 || pq.node >= p.nx * p.ny)
            bc->err = "assemble: gather index out of range";
        }
      }
      // below the top FP64 levels the mixed paths carry U, L and the Sigma
      // update in float-float (complex64 for Sigma only on request)
      const bool below_top = mixed && p.cl[op.cluster].depth > top_levels;
      const Arith ua = below_top ? kFF : kFP64;
      if (s > 0) {
        const int lc = (ff_all && below_top) ? 1 : 0;
        inv[lc].push_back(findgb::InvOp{M, escr, n, s, piv, escr * 4, ldl ? dv : nullptr});
        lv.inv_max[lc] = std::max(lv.inv_max[lc], s);
        lv.fl_inv[lc] += 8.0 * (double)s * s * s / 3.0;
        if (b > 0) {
          const int tc = below_top ? 1 : 0;
          findgb::TrsmOp t;
          t.M = M; t.estride = escr; t.ld = n; t.s = s; t.b = b;
          t.piv = piv; t.piv_estride = escr * 4;
          t.L = Lm; t.l_estride = escr;
          t.dv = ldl ? dv : nullptr;
          t.Wt = ldl ? Wt : nullptr;
          t.Yd = ldl ? Yd : nullptr;
          if (bc && ldl) {
            bc->block(Wt, b, s, s, escr, batch, "trsm W^T");
            bc->block(Yd, b, s, s, escr, batch, "trsm W^T D^-1");
            bc->block(dv, 1, 2 * s, 2 * s, escr, batch, "ldl D");
          }
          t.tile0 = (int)trs_map[tc].size();
          for (int r = 0; r < (b + lv.rb - 1) / lv.rb; ++r) trs_map[tc].push_back((int)trs.size());
          trs.push_back(t);
          lv.fl_trsm[tc] += 8.0 * (double)s * s * b;
          if (bc) bc->block(Lm, b, s, s, escr, batch, "trsm L");
        }
      }
      lv.by_asm += 16.0 * ((sig_op ? 2.0 : 1.0) * n * n + (double)a.d1 * a.d1 + (double)a.d2 * a.d2 +
                           (sig_op && a.r1 ? (double)a.d1 * a.d1 : 0.0) +
                           (sig_op && a.r2 ? (double)a.d2 * a.d2 : 0.0));
      // stage 0: U = M(B,B) - L M(S,B)                        (Eq. 2)
      findgb::GemmOp q = gemm0();
      q.m = b; q.n = b; q.k = s;
      if (ldl && s > 0) {
        // U = M(B,B) - (W^T D^-1) (W^T)^T, the symmetric form of Eq. 2 (Sec. 4.2)
        q.A = Yd; q.lda = s; q.sa = escr; q.alpha = -1.0;
        q.B = Wt; q.ldb = s; q.sb = escr; q.opb = 2;
      } else {
        q.A = Lm; q.lda = s; q.sa = escr; q.alpha = -1.0;
        q.B = M + s; q.ldb = n; q.sb = escr;
      }
      q.C = M + (int64_t)s * n + s; q.ldc = n; q.sc = escr; q.beta = 1.0;
      q.D = umat(op.dst); q.ldd = b; q.sd = (int64_t)b * b;
      q.sym = 1;  // U is complex symmetric when A is (Property 1)
      gemm_ok(q); route(q, 0, ua);
      const int c64_from = h->desc.sigma_c64_depth;
      const Arith sa = !below_top ? kFP64
                       : ((c64_from > 0 && p.cl[op.cluster].depth >= c64_from) ? kC64 : kFF);
      if (sig_op) {
        // stage 0: T = L Sigma(S,S) - Sigma(B,S)
        q = gemm0();
        q.m = b; q.n = s; q.k = s;
        q.A = Lm; q.lda = s; q.sa = escr;
        q.B = Sg; q.ldb = n; q.sb = escr;
        q.C = Sg + (int64_t)s * n; q.ldc = n; q.sc = escr; q.beta = -1.0;
        q.D = T; q.ldd = s; q.sd = escr;
        gemm_ok(q); route(q, 0, sa);
        // stage 1: R = Sigma(B,B) - L Sigma(S,B) + T L^H     (Eq. 7)
        q = gemm0();
        q.m = b; q.n = b; q.k = s; q.k2 = s;
        q.A = Lm; q.lda = s; q.sa = escr; q.alpha = -1.0;
        q.B = Sg + s; q.ldb = n; q.sb = escr;
        q.A2 = T; q.lda2 = s; q.sa2 = escr; q.alpha2 = 1.0;
        q.B2 = Lm; q.ldb2 = s; q.sb2 = escr; q.opb2 = 1;
        q.C = Sg + (int64_t)s * n + s; q.ldc = n; q.sc = escr; q.beta = 1.0;
        q.D = rmat(op.dst); q.ldd = b; q.sd = (int64_t)b * b;
        // R is anti-Hermitian in exact arithmetic, but its computed entries
        // carry cancellation errors that later steps rely on staying
        // mutually consistent: mirroring one triangle was measured to raise
        // the diag G< error from 1e-6 to 1e-2 (complex64) and from 5e-15 to
        // 3e-11 (FP64), so R is computed in full
        gemm_ok(q); route(q, 1, sa);
      }
    }
    lv.nops = (int)ops.size();
    lv.asmops = arx.put(asmops);
    lv.row_op = arx.put(row_op);
    for (int c = 0; c < 4; ++c) {
      lv.inv[c] = arx.put(inv[c]);
      lv.ninv[c] = (int)inv[c].size();
    }
    lv.trsm = arx.put(trs);
    for (int c = 0; c < 2; ++c) {
      lv.trsm_map[c] = arx.put(trs_map[c]);
      lv.ntrsm[c] = (int)trs_map[c].size();
    }
    lv.nstages = lesser ? 2 : 1;
    for (int k = 0; k < lv.nstages; ++k) {
      lv.st[k].ops = arx.put(g[k]);
      for (int c = 0; c < 6; ++c) {
        lv.st[k].map[c] = arx.put(maps[k][c]);
        lv.st[k].nmap[c] = (int)maps[k][c].size();
      }
    }
    finish_tc(lv, tcq, lv.nstages, off, arx, dry, need);
    lvx.push_back(lv);
  };

  // leaf level
  auto leaf_level = [&](Arena& arx, std::vector<Level>& lvx, bool dry, int64_t& need) {
    Level lv;
    lv.leaf = true;
    std::vector<findgb::AsmOp> asmops;
    std::vector<int> row_op;
    std::vector<findgb::InvOp> inv[4];
    std::vector<findgb::GemmOp> g[2];
    std::vector<int> maps[2][6];
    std::vector<findgb::TcOp> tcq[2];
    auto route = [&](const findgb::GemmOp& q, int k, Arith a) {
      const int nsl = tc_planes(h, q, a);
      if (nsl > 0 && q.m > 0 && q.n > 0) tcq[k].push_back(tc_from_gemm(q, nsl));
      else add_gemm(q, g[k], maps[k], &lv.st[k], a, small_max);
    };
    std::vector<findgb::ExtractOp> ext;
    int64_t off = 0;
    for (const auto& op : p.leaf_ops) {
      const int64_t slot = leaf_slot_elems(op, lesser);
      cplx* M = S0 + off;  // energy e at M + e * escr
      cplx* Sg = M + (int64_t)op.n * op.n;
      cplx* P = M + 2 * (int64_t)op.n * op.n;
      cplx* Q = P + (int64_t)op.c * op.n;
      off += slot;
      const int n = op.n;
      findgb::AsmOp a;
      a.n = n;
      a.row0 = lv.nrows;
      a.pos = op.pos;
      a.u1 = umat(op.src); a.r1 = rsrc(op.src); a.d1 = op.src < 0 ? 0 : p.mat_dim[op.src];
      a.u2 = nullptr; a.r2 = nullptr; a.d2 = 0;
      a.M = M;
      a.estride = escr;
      a.sig = lesser ? 1 : 0;
      for (int r = 0; r < n; ++r) row_op.push_back((int)asmops.size());
      lv.nrows += n;
      asmops.push_back(a);
      if (bc) {
        bc->block(M, lesser ? 2 * (int64_t)n + 2 * op.c : n, n, n, escr, batch, "leaf scratch");
        if (a.u1) bc->block(a.u1, a.d1, a.d1, a.d1, (int64_t)a.d1 * a.d1, batch, "leaf U");
        if (a.r1) bc->block(a.r1, a.d1, a.d1, a.d1, (int64_t)a.d1 * a.d1, batch, "leaf R");
        for (int q = 0; q < n && bc->err.empty(); ++q) {
          const findgb::Pos& pq = p.pos[op.pos + q];
          int d = pq.src == 1 ? a.d1 : 1;
          if (pq.src == 2 || pq.idx < 0 || pq.idx >= d || pq.node < 0 || pq.node >= p.nx * p.ny)
            bc->err = "leaf assemble: gather index out of range";
        }
        for (int b = 0; b < op.nbond && bc->err.empty(); ++b) {
          const findgb::LeafBond& lb = p.bonds[op.bond + b];
          if (lb.pi < op.nb || lb.pi >= n || lb.pj < 0 || lb.pj >= n || lb.bond < 0 || lb.bond >= p.n_bonds)
            bc->err = "leaf bond index out of range";
        }
      }
      {
        const bool leaf_ff = ff_all && p.cl[op.cluster].depth > top_levels;
        const int lc = (leaf_ff ? 1 : 0) + (n <= inv_smem ? 2 : 0);
        inv[lc].push_back(findgb::InvOp{M, escr, n, n, nullptr, 0});
        lv.inv_max[lc] = std::max(lv.inv_max[lc], n);
        lv.fl_inv[lc] += 8.0 * (double)n * n * n;
      }
      lv.max_s = std::max(lv.max_s, n);
      lv.by_asm += 16.0 * ((lesser ? 2.0 : 1.0) * n * n + (lesser ? 2.0 : 1.0) * (double)a.d1 * a.d1);
      lv.by_ext += 16.0 * (lesser ? 2.0 : 1.0) * op.c + (lesser ? 24.0 * op.nbond : 0.0);
      if (lesser) {
        // P = G_K(C, :) Sigma_K
        // Sigma< sparsity (Sec. 4.3): a leaf with no contact node has
        // Sigma_K = [R_Cbar 0; 0 0], so only the first nb columns of P are
        // nonzero and both products run over K = nb
        const bool zc = !h->sig_dense_build && op.nb > 0 && p.cl[op.cluster].y0 > 0 &&
                        p.cl[op.cluster].y1 < p.ny;
        const int kk = zc ? op.nb : n;
        findgb::GemmOp q = gemm0();
        q.m = op.c; q.n = kk; q.k = kk;
        q.A = M + (int64_t)op.nb * n; q.lda = n; q.sa = escr;
        q.B = Sg; q.ldb = n; q.sb = escr;
        q.D = P; q.ldd = n; q.sd = escr;
        // the leaf products G_K Sigma_K G_K^H carry diag G< directly: float-float
        // keeps the mixed paths' G< error near that of the complex64 Sigma
        // update alone (complex64 here reached 1e-5 on a 64x128 mesh)
        const Arith la = (mixed && p.cl[op.cluster].depth > top_levels) ? kFF : kFP64;
        gemm_ok(q); route(q, 0, la);
        // Q = P G_K^H = G<_K(C, :)
        q = gemm0();
        q.m = op.c; q.n = n; q.k = kk;
        q.A = P; q.lda = n; q.sa = escr;
        q.B = M; q.ldb = n; q.sb = escr; q.opb = 1;
        q.D = Q; q.ldd = n; q.sd = escr;
        gemm_ok(q); route(q, 1, la);
      }
      findgb::ExtractOp x;
      x.K = M;
      x.Q = lesser ? Q : nullptr;
      x.estride = escr;
      x.n = n; x.nb = op.nb; x.c = op.c;
      x.x0 = op.x0; x.y0 = op.y0; x.wx = op.wx;
      x.bond = op.bond; x.nbond = op.nbond;
      ext.push_back(x);
    }
    lv.nops = (int)p.leaf_ops.size();
    lv.asmops = arx.put(asmops);
    lv.row_op = arx.put(row_op);
    for (int c = 0; c < 4; ++c) {
      lv.inv[c] = arx.put(inv[c]);
      lv.ninv[c] = (int)inv[c].size();
    }
    lv.ext = arx.put(ext);
    lv.nstages = lesser ? 2 : 0;
    for (int k = 0; k < lv.nstages; ++k) {
      lv.st[k].ops = arx.put(g[k]);
      for (int c = 0; c < 6; ++c) {
        lv.st[k].map[c] = arx.put(maps[k][c]);
        lv.st[k].nmap[c] = (int)maps[k][c].size();
      }
    }
    finish_tc(lv, tcq, lv.nstages, off, arx, dry, need);
    lvx.push_back(lv);
  };

  auto build_all = [&](Arena& arx, std::vector<Level>& lvx, bool dry, int64_t& need) {
    lvx.clear();
    for (const auto& lv : p.up_levels) elim_level(lv, arx, lvx, dry, need);
    h->n_up = (int)p.up_levels.size();
    for (const auto& lv : p.dn_levels) elim_level(lv, arx, lvx, dry, need);
    h->n_dn = (int)p.dn_levels.size();
    leaf_level(arx, lvx, dry, need);
  };
  {
    int64_t need = 0;
    Arena a0;
    std::vector<Level> l0;
    Bounds* const bc_real = bc;  // the dry build's pointers use a provisional escr
    bc = nullptr;
    build_all(a0, l0, true, need);
    bc = bc_real;
    escr = (std::max(escr, need) + 63) & ~int64_t(63);
  }
  int64_t need = 0;
  build_all(ar_out, levels_out, false, need);
  scratch_elems = escr;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Computes the workspace layout for (batch, lesser); meta_bytes is the size
// of the descriptor arena.
Layout make_layout(const find_handle* h, int batch, bool lesser, int64_t scratch_elems,
                   size_t meta_bytes) {
  const findgb::Plan& p = h->plan;
  const size_t n = (size_t)p.nx * p.ny, nx = p.nx, c16 = sizeof(cplx);
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  L.V = take(n * 8);
  L.phi = take(nx * nx * 8);
  L.eps = take(nx * 8);
  L.tau = take(nx * 8);
  L.E = take(batch * c16);
  L.sigL = take(batch * nx * nx * c16);
  L.sigR = take(batch * nx * nx * c16);
  L.modes = take(batch * nx * c16);
  L.dles = take(lesser ? batch * n * c16 : 0);
  L.U = take((size_t)p.mat_elems * batch * c16);
  L.R = take(lesser ? (size_t)p.mat_elems * batch * c16 : 0);
  L.scratch = take((size_t)scratch_elems * batch * c16);
  L.oG = take(batch * n * c16);
  L.oGl = take(lesser ? batch * n * c16 : 0);
  L.oJ = take(lesser ? batch * (size_t)p.n_bonds * 8 : 0);
  L.pos = take(p.pos.size() * sizeof(findgb::Pos));
  L.bonds = take(p.bonds.size() * sizeof(findgb::LeafBond));
  L.status = take(256);
  L.meta = take(meta_bytes);
  L.total = o;
  return L;
}

// The FP64 path eliminates by LDL^T (Sec. 4.2) unless FIND_FLAG_LU asks for
// the LU; the mixed paths by LU unless FIND_FLAG_LDL asks for LDL^T.  A call
// can use LDL^T only when A = A^T, i.e. with the closed-form lead
// self-energies (Phi diag(sigma) Phi^T); a caller's Sigma takes the LU.
bool default_ldl(const find_handle* h) {
  if (h->desc.flags & FIND_FLAG_LU) return false;
  return h->desc.precision == FIND_FP64 || (h->desc.flags & FIND_FLAG_LDL);
}

double workspace_bytes(find_handle* h, int batch, bool lesser, std::string* check_err = nullptr,
                       int ldl = -1) {
  h->ldl_build = ldl < 0 ? default_ldl(h) : ldl != 0;
  h->sig_dense_build = false;
  Arena ar;
  std::vector<Level> lv;
  int64_t se = 0;
  Layout L0 = make_layout(h, batch, lesser, 0, 0);
  build_tables(h, nullptr, L0, batch, lesser, ar, lv, se);
  Layout L = make_layout(h, batch, lesser, se, ar.buf.size());
  if (check_err) {
    // the same bounds check as before an upload, against a synthetic base
    // address (nothing is dereferenced)
    unsigned char* fake = reinterpret_cast<unsigned char*>(uintptr_t(1) << 40);
    Arena a2;
    Bounds bc;
    bc.lo = fake;
    bc.hi = fake + L.meta;
    bc.s_lo = fake + L.scratch;
    bc.s_hi = fake + L.scratch + (size_t)se * batch * sizeof(cplx);
    bc.s_stride = se * (int64_t)sizeof(cplx);
    build_tables(h, fake, L, batch, lesser, a2, lv, se, &bc);
    *check_err = bc.err;
  }
  return (double)L.total;
}

// Captured passes hold pointers into the workspace: drop them with it.
void drop_graphs(find_handle* h) {
  for (auto& g : h->graphs) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

void release(find_handle* h) {
  drop_graphs(h);
  if (h->rgf_ws) cudaFree(h->rgf_ws);
  h->rgf_ws = nullptr;
  h->rgf_batch = 0;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->batch = 0;
  h->lesser = -1;
  h->levels.clear();
}

// dense_sig: the call passes a node-diagonal Sigma<, so no cluster may skip
// its Sigma update; tables built that way serve every later call too.
int ensure_workspace(find_handle* h, int batch, bool lesser, bool ldl, bool dense_sig = false) {
  if (h->ws && h->batch >= batch && (h->lesser == 1 || !lesser) && h->ldl == ldl &&
      (!dense_sig || h->sig_dense))
    return FIND_OK;
  release(h);
  h->ldl_build = ldl;
  h->sig_dense_build = dense_sig;
  Arena ar;
  std::vector<Level> lv;
  int64_t se = 0;
  Layout L0 = make_layout(h, batch, lesser, 0, 0);
  build_tables(h, nullptr, L0, batch, lesser, ar, lv, se);
  Layout L = make_layout(h, batch, lesser, se, ar.buf.size());
  unsigned char* ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, L.total);
  if (e != cudaSuccess) return cuda_fail(h, e, "workspace allocation");
  h->ws = ws;
  h->lay = L;
  h->batch = batch;
  h->lesser = lesser ? 1 : 0;
  h->ldl = ldl;
  h->sig_dense = dense_sig;
  Arena real;
  Bounds bc;
  bc.lo = ws;
  bc.hi = ws + L.meta;
  bc.s_lo = ws + L.scratch;
  bc.s_hi = ws + L.scratch + (size_t)se * batch * sizeof(cplx);
  bc.s_stride = se * (int64_t)sizeof(cplx);
  int map_err = 0;
  build_tables(h, ws, L, batch, lesser, real, h->levels, se, &bc, &map_err);
  if (!bc.err.empty()) {
    release(h);
    return fail(h, FIND_EINVAL, "internal table check failed: " + bc.err);
  }
  if (map_err) {
    release(h);
    return fail(h, FIND_ECUDA, "tensor map encoding of the digit planes failed");
  }
  const findgb::Plan& p = h->plan;
  e = cudaMemcpy(ws + L.V, h->V.data(), h->V.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ws + L.phi, h->phi.data(), h->phi.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ws + L.eps, h->eps.data(), h->eps.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ws + L.tau, h->tau.data(), h->tau.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(ws + L.pos, p.pos.data(), p.pos.size() * sizeof(findgb::Pos), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !p.bonds.empty())
    e = cudaMemcpy(ws + L.bonds, p.bonds.data(), p.bonds.size() * sizeof(findgb::LeafBond),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(ws + L.meta, real.buf.data(), real.buf.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    release(h);
    return cuda_fail(h, e, "workspace upload");
  }
  return FIND_OK;
}

int choose_batch(find_handle* h, int nE, bool lesser, bool ldl) {
  if (h->desc.max_batch > 0) return std::min(h->desc.max_batch, nE);
  size_t fr = 0, tot = 0;
  if (h->ws && h->lesser >= (lesser ? 1 : 0) && h->ldl == ldl) return std::min(h->batch, nE);
  if (h->ws && h->ldl != ldl) release(h);  // the other elimination's tables: free them first
  cudaMemGetInfo(&fr, &tot);
  double one = workspace_bytes(h, 1, lesser, nullptr, ldl);
  double two = workspace_bytes(h, 2, lesser, nullptr, ldl);
  double per = std::max(1.0, two - one);
  double budget = 0.70 * (double)fr - (one - per);
  int b = (int)std::floor(budget / per);
  return std::max(1, std::min({b, 64, nE}));
}

template <class T>
const T* at(const find_handle* h, size_t off) {
  return reinterpret_cast<const T*>(h->ws + h->lay.meta + off);
}

const int kClasses = 19;
const char* kClassNames[kClasses] = {"lead",     "assemble", "invert",  "lu",   "trsm",
                                     "zgemm32",  "zgemm64",  "extract", "cgemm32", "cgemm64",
                                     "ffgemm32", "ffgemm64", "fftrsm",  "fflu", "ffinvert",
                                     "tcsplit",  "tcgemm", "ldl",     "ffldl"};
// profiler class of each GEMM launch class 2 * arith + big
const int kGemmClass[6] = {5, 6, 8, 9, 10, 11};

// 1 when the TRSM launch of class c (1: float-float) reads factors that the
// float-float LU left as float-float words: on FIND_MIXED_FF the LU and the
// TRSM of a level share their class; on FIND_MIXED the LU is always FP64.
int ff_factors(const find_handle* h, int c) {
  return (c == 1 && h->desc.precision == FIND_MIXED_FF) ? 1 : 0;
}

// 1 when every U update runs on one triangle (closed-form leads make
// A = A^T): by default on the mixed paths only, see FIND_FLAG_SYM_U.
int sym_updates(const find_handle* h, const void* sigL, const void* sigR) {
  if (sigL || sigR || (h->desc.flags & FIND_FLAG_FULL_U)) return 0;
  if (h->desc.precision == FIND_FP64 && !(h->desc.flags & FIND_FLAG_SYM_U)) return 0;
  return 1;
}

cudaEvent_t take_event(find_handle* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Runs `launch` on stream st; while profiling, brackets it with events.
template <class F>
void timed(find_handle* h, cudaStream_t st, int cls, double flops, double bytes, F&& launch) {
  if (!h->prof) {
    launch();
    return;
  }
  cudaEvent_t a = take_event(h), b = take_event(h);
  cudaEventRecord(a, st);
  launch();
  cudaEventRecord(b, st);
  h->pending.push_back(find_handle::Pending{cls, a, b, flops, bytes});
}

void run_level(find_handle* h, const Level& lv, const findgb::DevProblem& P, bool lesser,
               int e_base, int nb, cudaStream_t st, cplx* oG, cplx* oGl, double* oJ,
               int want_bonds, int e_off = 0, int sym_mask = 0) {
  const Layout& L = h->lay;
  auto pos = reinterpret_cast<const findgb::Pos*>(h->ws + L.pos);
  int* status = reinterpret_cast<int*>(h->ws + L.status);
  timed(h, st, 1, 0.0, lv.by_asm * nb, [&] {
    findgb::launch_assemble(at<findgb::AsmOp>(h, lv.asmops), at<int>(h, lv.row_op), lv.nrows, pos,
                            P, lesser ? 1 : 0, nb, st, e_off);
  });
  if (lv.leaf) {
    for (int c = 0; c < 4; ++c)
      if (lv.ninv[c] > 0)
        timed(h, st, (c & 1) ? 14 : 2, lv.fl_inv[c] * nb, 0.0, [&] {
          findgb::launch_invert(at<findgb::InvOp>(h, lv.inv[c]), lv.ninv[c], lv.inv_max[c], status,
                                e_base, nb, st, e_off, c & 1, c >> 1);
        });
  } else {
    for (int c = 0; c < 2; ++c)
      if (lv.ninv[c] > 0) {
        const bool ldl = h->ldl;  // LDL^T: half the flops of the LU
        timed(h, st, ldl ? (c ? 18 : 17) : (c ? 13 : 3), lv.fl_inv[c] * (ldl ? 0.5 : 1.0) * nb, 0.0, [&] {
          if (ldl)
            findgb::launch_ldl(at<findgb::InvOp>(h, lv.inv[c]), lv.ninv[c], lv.inv_max[c], status, e_base,
                               nb, st, e_off, c);
          else
            findgb::launch_lu(at<findgb::InvOp>(h, lv.inv[c]), lv.ninv[c], lv.inv_max[c], status, e_base,
                              nb, st, e_off, c);
        });
      }
    for (int c = 0; c < 2; ++c)
      if (lv.ntrsm[c] > 0)
        timed(h, st, c ? 12 : 4, lv.fl_trsm[c] * nb, 0.0, [&] {
          findgb::launch_trsm(at<findgb::TrsmOp>(h, lv.trsm), at<int>(h, lv.trsm_map[c]), lv.ntrsm[c],
                              lv.rb, lv.max_s, nb, st, c, e_off, h->ldl ? 0 : ff_factors(h, c), h->ldl);
        });
  }
  for (int k = 0; k < lv.nstages; ++k) {
    const Stage& s = lv.st[k];
    const findgb::GemmOp* ops = at<findgb::GemmOp>(h, s.ops);
    for (int c = 0; c < 6; ++c)
      if (s.nmap[c])
        timed(h, st, kGemmClass[c], ((sym_mask & 1) ? s.fl_sym[c] : s.fl[c]) * nb, 0.0, [&] {
          findgb::launch_gemm(ops, at<int>(h, s.map[c]), s.nmap[c], c & 1, nb, st, c >> 1, e_off,
                              sym_mask);
        });
    for (const TcChunk& c : s.tc) {
      const findgb::TcOp* tops = at<findgb::TcOp>(h, c.ops);
      timed(h, st, 15, 0.0, c.by * nb, [&] {
        findgb::launch_tc_split(c.L, tops, at<int4>(h, c.sitems), c.nsitems, at<int4>(h, c.ritems),
                                c.nritems, at<int4>(h, c.citems), c.ncitems, nb, st, e_off);
      });
      timed(h, st, 16, c.fl * nb, 0.0, [&] {
        findgb::launch_tc_mma(c.L, tops, at<int>(h, c.tmap), c.ntiles, status, nb, st, e_off);
      });
    }
  }
  if (lv.leaf)
    timed(h, st, 7, 0.0, lv.by_ext * nb, [&] {
      findgb::launch_extract(at<findgb::ExtractOp>(h, lv.ext), lv.nops,
                             reinterpret_cast<const findgb::LeafBond*>(h->ws + L.bonds), P,
                             lesser ? 1 : 0, want_bonds, oG, oGl, oJ,
                             (int64_t)h->plan.nx * h->plan.ny, h->plan.n_bonds, nb, st, e_off);
    });
}

// Streams and events of the concurrent energy groups, created once per
// handle: kMaxGroups streams, one join event per group and the fork event
// at index kMaxGroups.
constexpr int kMaxGroups = 4;

int ensure_group_streams(find_handle* h) {
  while ((int)h->gstreams.size() < kMaxGroups) {
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "group stream");
    h->gstreams.push_back(s);
  }
  while ((int)h->gevents.size() < kMaxGroups + 1) {
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "group event");
    h->gevents.push_back(ev);
  }
  return FIND_OK;
}

int solve(find_handle* h, const double* E, int nE, const double* sigL, const double* sigR,
          double fL, double fR, const double* dles, int dles_per_e, double* G, double* Gl,
          double* J, void* stream, bool lesser) {
  if (!h) return fail(nullptr, FIND_EINVAL, "null handle");
  if (nE < 0) return fail(h, FIND_EINVAL, "nE < 0");
  if (nE == 0) return FIND_OK;
  if (!E || !G || (lesser && !Gl)) return fail(h, FIND_EINVAL, "E and the diag outputs must not be NULL");
  DeviceGuard guard(h->desc.device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const findgb::Plan& p = h->plan;
  const int64_t n = (int64_t)p.nx * p.ny, nx = p.nx;
  const bool ldl = default_ldl(h) && !sigL && !sigR;
  int batch = choose_batch(h, nE, lesser, ldl);
  int rc = ensure_workspace(h, batch, lesser, ldl, lesser && dles != nullptr);
  if (rc != FIND_OK) return rc;
  batch = std::min(batch, h->batch);
  const Layout& L = h->lay;
  unsigned char* ws = h->ws;
  cplx* dE = reinterpret_cast<cplx*>(ws + L.E);
  cplx* dsL = reinterpret_cast<cplx*>(ws + L.sigL);
  cplx* dsR = reinterpret_cast<cplx*>(ws + L.sigR);
  cplx* dmodes = reinterpret_cast<cplx*>(ws + L.modes);
  cplx* ddl = reinterpret_cast<cplx*>(ws + L.dles);
  int* status = reinterpret_cast<int*>(ws + L.status);
  // graph mode writes every output to the workspace's staging buffers (the
  // captured launches must not hold the caller's pointers) and copies out
  const bool graph = (h->desc.flags & FIND_FLAG_GRAPH) != 0;
  const bool dG = !graph && device_accessible(G);
  const bool dGl = !lesser || (!graph && device_accessible(Gl));
  const bool dJ = !lesser || !J || (!graph && device_accessible(J));
  const int want_bonds = (lesser && J) ? 1 : 0;
  if (graph) {
    int rc2 = ensure_group_streams(h);
    if (rc2 != FIND_OK) return rc2;
    if (!h->cap_stream) {
      cudaError_t ce = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
      if (ce != cudaSuccess) return cuda_fail(h, ce, "capture stream");
    }
  }

  cudaError_t e = cudaMemsetAsync(status, 0x7f, 2 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  const int kNoError = 0x7f7f7f7f;
  if (lesser && dles && !dles_per_e) {
    e = cudaMemcpyAsync(ddl, dles, n * sizeof(cplx), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "sigma_lesser_diag copy");
  }
  for (int e0 = 0; e0 < nE; e0 += batch) {
    const int nb = std::min(batch, nE - e0);
    e = cudaMemcpyAsync(dE, E + 2 * (int64_t)e0, nb * sizeof(cplx), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy copy");
    const cplx* useL = dsL;
    const cplx* useR = dsR;
    if (!sigL && !sigR) useR = dsL;
    if (sigL) {
      e = cudaMemcpyAsync(dsL, sigL + 2 * (int64_t)e0 * nx * nx, nb * nx * nx * sizeof(cplx),
                          cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "sigmaL copy");
      if (!sigR) useR = dsR;
    }
    if (sigR) {
      e = cudaMemcpyAsync(dsR, sigR + 2 * (int64_t)e0 * nx * nx, nb * nx * nx * sizeof(cplx),
                          cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "sigmaR copy");
    }
    if (!sigL && sigR) useL = dsL;
    findgb::DevProblem P;
    P.nx = p.nx; P.ny = p.ny; P.stencil = p.stencil;
    P.t = h->desc.t; P.tp = h->desc.tp; P.onsite0 = h->desc.onsite0;
    P.V = reinterpret_cast<const double*>(ws + L.V);
    P.E = dE; P.sigL = useL; P.sigR = useR;
    P.fL = fL; P.fR = fR;
    P.dles = nullptr; P.dles_estride = 0;
    if (lesser && dles) {
      P.dles = ddl;
      if (dles_per_e) {
        P.dles_estride = n;
        e = cudaMemcpyAsync(ddl, dles + 2 * (int64_t)e0 * n, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "sigma_lesser_diag copy");
      }
    }
    cplx* oG = dG ? reinterpret_cast<cplx*>(G) + (int64_t)e0 * n : reinterpret_cast<cplx*>(ws + L.oG);
    cplx* oGl = lesser ? (dGl ? reinterpret_cast<cplx*>(Gl) + (int64_t)e0 * n
                              : reinterpret_cast<cplx*>(ws + L.oGl))
                       : nullptr;
    double* oJ = want_bonds ? (dJ ? J + (int64_t)e0 * p.n_bonds : reinterpret_cast<double*>(ws + L.oJ))
                            : nullptr;
    // A = A^T when both leads take the closed form (Phi diag(sigma) Phi^T):
    // then every U is complex symmetric and its update may run on one triangle
    const int sym_mask = sym_updates(h, sigL, sigR);
    // the device work of one pass: closed-form lead Sigma, then every level;
    // independent energy groups on their own streams, so that one group's
    // low-parallelism phases (LU of the few large top blocks) overlap other
    // groups' work
    auto pass = [&](cudaStream_t qs) -> int {
      if (!sigL || !sigR) {
        cplx* dst = !sigL ? dsL : dsR;
        timed(h, qs, 0, 2.0 * nx * nx * nx * nb, 0.0, [&] {
          findgb::launch_lead_modes(dE, nb, reinterpret_cast<const double*>(ws + L.eps),
                                    reinterpret_cast<const double*>(ws + L.tau), (int)nx, dmodes, qs);
          findgb::launch_lead_dense(dmodes, reinterpret_cast<const double*>(ws + L.phi), (int)nx, nb,
                                    dst, qs);
        });
      }
      const int gsz = h->desc.energy_group > 0 ? h->desc.energy_group : 8;
      const int ng = std::min((nb + gsz - 1) / gsz, kMaxGroups);
      if (ng <= 1) {
        for (const Level& lv : h->levels)
          run_level(h, lv, P, lesser, e0, nb, qs, oG, oGl, oJ, want_bonds, 0, sym_mask);
        return FIND_OK;
      }
      int rc2 = ensure_group_streams(h);
      if (rc2 != FIND_OK) return rc2;
      cudaEvent_t fork = h->gevents[kMaxGroups];
      cudaEventRecord(fork, qs);
      const int per = (nb + ng - 1) / ng;
      for (int g = 0; g < ng; ++g) {
        const int lo = g * per, cnt = std::min(per, nb - lo);
        if (cnt <= 0) continue;
        cudaStream_t gs = h->gstreams[g];
        cudaStreamWaitEvent(gs, fork, 0);
        for (const Level& lv : h->levels)
          run_level(h, lv, P, lesser, e0, cnt, gs, oG, oGl, oJ, want_bonds, lo, sym_mask);
        cudaEventRecord(h->gevents[g], gs);
        cudaStreamWaitEvent(qs, h->gevents[g], 0);
      }
      return FIND_OK;
    };
    if (!graph) {
      int rc2 = pass(st);
      if (rc2 != FIND_OK) return rc2;
    } else {
      const find_handle::GraphKey key{nb, e0, lesser ? 1 : 0, want_bonds, sigL ? 1 : 0, sigR ? 1 : 0,
                                      dles ? 1 : 0, dles_per_e, sym_mask, fL, fR};
      cudaGraphExec_t exec = nullptr;
      for (size_t i = 0; i < h->graphs.size(); ++i)
        if (h->graphs[i].key == key) {
          find_handle::Graph g = h->graphs[i];
          h->graphs.erase(h->graphs.begin() + i);
          h->graphs.push_back(g);
          exec = g.exec;
          break;
        }
      if (!exec) {
        // the event profiler's records cannot live inside a graph
        const bool prof = h->prof;
        h->prof = false;
        e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
          h->prof = prof;
          return cuda_fail(h, e, "begin capture");
        }
        int rc2 = pass(h->cap_stream);
        cudaGraph_t gr = nullptr;
        e = cudaStreamEndCapture(h->cap_stream, &gr);
        h->prof = prof;
        if (rc2 != FIND_OK) {
          if (gr) cudaGraphDestroy(gr);
          return rc2;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
        e = cudaGraphInstantiate(&exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(h, e, "graph instantiate");
        if (h->graphs.size() >= 8) {
          cudaGraphExecDestroy(h->graphs.front().exec);
          h->graphs.erase(h->graphs.begin());
        }
        h->graphs.push_back(find_handle::Graph{key, exec});
      }
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    if (!dG) {
      e = cudaMemcpyAsync(G + 2 * (int64_t)e0 * n, oG, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "diagG copy-out");
    }
    if (lesser && !dGl) {
      e = cudaMemcpyAsync(Gl + 2 * (int64_t)e0 * n, oGl, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "diagGl copy-out");
    }
    if (want_bonds && !dJ) {
      e = cudaMemcpyAsync(J + (int64_t)e0 * p.n_bonds, oJ, nb * (size_t)p.n_bonds * 8, cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "bond current copy-out");
    }
  }
  int hs2[2] = {kNoError, kNoError};
  e = cudaMemcpyAsync(hs2, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve");
  if (hs2[1] != kNoError) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "a bounded wait of the tensor-core product ran out (role %d)", hs2[1]);
    return fail(h, FIND_ETIMEOUT, buf);
  }
  const int hs = hs2[0];
  if (hs != kNoError) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "exactly zero pivot at energy index %d", hs);
    return fail(h, FIND_ESINGULAR, buf);
  }
  h->err.clear();
  return FIND_OK;
}

// ---------------------------------------------------------------- RGF baseline
// The recursive Green's function method over the Ny transport slices, FP64,
// all energies of a pass in lockstep:
//   right-connected sweep  gR_y = (A_yy - C gR_{y+1} C)^-1, y = Ny-1 .. 0
//   first column           G_00 = gR_0, G_y0 = -gR_y C G_{y-1,0}
//   left-connected sweep   gL_y = (A_yy - C gL_{y-1} C)^-1, y = 0 .. Ny-1
//   backward               G_yy = gL_y + gL_y C G_{y+1,y+1} C gL_y,
//                          G_{y,N-1} = -gL_y C G_{y+1,N-1}
//   diag G<_yy = diag(G_y0 S<_L G_y0^H) + diag(G_{y,N-1} S<_R G_{y,N-1}^H)
// (Sigma< on the contact slices only).  Storage per energy: gR and gL of
// every slice, and nine Nx x Nx working blocks.
namespace {

// Layout of the RGF workspace for `batch` energies (byte offsets).
struct RgfLayout {
  size_t est = 0;                       // complex entries per energy in the block area
  size_t blk, V, phi, eps, tau, E, sig, modes, SL, SR, G, Gl, stat, meta, total;
};

RgfLayout rgf_layout(const find_handle* h, int batch, size_t meta_bytes) {
  const int nx = h->plan.nx, ny = h->plan.ny;
  const size_t b2 = (size_t)nx * nx, c16 = sizeof(cplx);
  RgfLayout L;
  L.est = ((2 * (size_t)ny + 9) * b2 + 15) & ~size_t(15);  // gR[ny], gL[ny], G0 x2, GN x2, D x2, W, T, X
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
  L.blk = take(L.est * batch * c16);
  L.V = take((size_t)nx * ny * 8);
  L.phi = take(b2 * 8);
  L.eps = take((size_t)nx * 8);
  L.tau = take((size_t)nx * 8);
  L.E = take(batch * c16);
  L.sig = take(batch * b2 * c16);
  L.modes = take(batch * (size_t)nx * c16);
  L.SL = take(batch * b2 * c16);
  L.SR = take(batch * b2 * c16);
  L.G = take(batch * (size_t)nx * ny * c16);
  L.Gl = take(batch * (size_t)nx * ny * c16);
  L.stat = take(256);
  L.meta = take(meta_bytes);
  L.total = o;
  return L;
}

// The GEMM and inversion descriptors of one RGF pass against `base` (in the
// order rgf_run consumes them), written into `ar`.
void rgf_build(const find_handle* h, unsigned char* base, const RgfLayout& L, Arena& ar,
               size_t* og, size_t* oi, size_t* oz) {
  const int nx = h->plan.nx, ny = h->plan.ny;
  const size_t b2 = (size_t)nx * nx;
  const int64_t es = (int64_t)L.est;
  cplx* B0 = reinterpret_cast<cplx*>(base + L.blk);
  auto blk = [&](size_t k) { return B0 + k * b2; };
  const size_t wk = 2 * (size_t)ny;
  cplx* G0[2] = {blk(wk), blk(wk + 1)};
  cplx* GN[2] = {blk(wk + 2), blk(wk + 3)};
  cplx* D[2] = {blk(wk + 4), blk(wk + 5)};
  cplx* Wb = blk(wk + 6);
  cplx* Tb = blk(wk + 7);
  cplx* Xb = blk(wk + 8);
  cplx* SL = reinterpret_cast<cplx*>(base + L.SL);
  cplx* SR = reinterpret_cast<cplx*>(base + L.SR);
  std::vector<findgb::GemmOp> g;
  std::vector<findgb::InvOp> inv;
  auto mm = [&](const cplx* A, const cplx* B, int64_t sb, const cplx* C, cplx* Dd, double alpha) {
    findgb::GemmOp q = gemm0();
    q.m = nx; q.n = nx; q.k = nx;
    q.A = A; q.lda = nx; q.sa = es; q.alpha = alpha;
    q.B = B; q.ldb = nx; q.sb = sb;
    if (C) { q.C = C; q.ldc = nx; q.sc = es; q.beta = 1.0; }
    q.D = Dd; q.ldd = nx; q.sd = es;
    q.tiles_n = (nx + 63) / 64;
    g.push_back(q);
  };
  for (int y = 0; y < ny; ++y) {
    inv.push_back(findgb::InvOp{blk(y), es, nx, nx, nullptr, 0, nullptr});            // gR_y
    inv.push_back(findgb::InvOp{blk((size_t)ny + y), es, nx, nx, nullptr, 0, nullptr}); // gL_y
  }
  // column pass, op 2y: G_y0 = -gR_y W;  op 2y+1: X = G_y0 S<_L
  for (int y = 0; y < ny; ++y) {
    mm(blk(y), Wb, es, nullptr, G0[y & 1], -1.0);
    mm(y == 0 ? blk(0) : G0[y & 1], SL, (int64_t)b2, nullptr, Xb, 1.0);
  }
  // backward, op 2ny + 4y .. +3: T = gL_y Q; D_y = gL_y + T gL_y; GN_y = -gL_y W;
  // X = GN_y S<_R (GN_{ny-1} = gL_{ny-1})
  for (int y = 0; y < ny; ++y) {
    cplx* gl = blk((size_t)ny + y);
    mm(gl, Wb, es, nullptr, Tb, 1.0);
    mm(Tb, gl, es, gl, D[y & 1], 1.0);
    mm(gl, Wb, es, nullptr, GN[y & 1], -1.0);
    mm(y == ny - 1 ? gl : GN[y & 1], SR, (int64_t)b2, nullptr, Xb, 1.0);
  }
  *og = ar.put(g);
  *oi = ar.put(inv);
  std::vector<int> zmap((size_t)((nx + 63) / 64) * ((nx + 63) / 64), 0);
  *oz = ar.put(zmap);
}

int rgf_solve(find_handle* h, const double* E, int nE, double fL, double fR, double* G, double* Gl,
              void* stream) {
  if (!h) return fail(nullptr, FIND_EINVAL, "null handle");
  if (nE < 0) return fail(h, FIND_EINVAL, "nE < 0");
  if (nE == 0) return FIND_OK;
  if (!E || !G || !Gl) return fail(h, FIND_EINVAL, "E, diagG and diagGl must not be NULL");
  DeviceGuard guard(h->desc.device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const findgb::Plan& p = h->plan;
  const int nx = p.nx, ny = p.ny;
  const int64_t n = (int64_t)nx * ny;
  const size_t b2 = (size_t)nx * nx;
  int batch = h->desc.max_batch > 0 ? std::min(h->desc.max_batch, nE) : 0;
  if (batch == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    if (h->rgf_ws) fr += rgf_layout(h, h->rgf_batch, h->rgf_meta_bytes).total;
    const double per = (double)(rgf_layout(h, 2, 0).total - rgf_layout(h, 1, 0).total);
    batch = std::max(1, std::min({(int)(0.6 * (double)fr / per), 64, nE}));
  }
  if (!h->rgf_ws || h->rgf_batch < batch) {
    if (h->rgf_ws) cudaFree(h->rgf_ws);
    h->rgf_ws = nullptr;
    Arena sizing;
    size_t t3[3];
    rgf_build(h, nullptr, rgf_layout(h, batch, 0), sizing, &t3[0], &t3[1], &t3[2]);
    const RgfLayout L = rgf_layout(h, batch, sizing.buf.size());
    unsigned char* base = nullptr;
    cudaError_t e = cudaMalloc(&base, L.total);
    if (e != cudaSuccess) return cuda_fail(h, e, "RGF workspace allocation");
    Arena real;
    rgf_build(h, base, L, real, &h->rgf_tab[0], &h->rgf_tab[1], &h->rgf_tab[2]);
    e = cudaMemcpy(base + L.V, h->V.data(), h->V.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + L.phi, h->phi.data(), h->phi.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + L.eps, h->eps.data(), h->eps.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + L.tau, h->tau.data(), h->tau.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + L.meta, real.buf.data(), real.buf.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(base);
      return cuda_fail(h, e, "RGF workspace upload");
    }
    h->rgf_ws = base;
    h->rgf_batch = batch;
    h->rgf_meta_bytes = sizing.buf.size();
  }
  batch = std::min(batch, h->rgf_batch);
  const RgfLayout L = rgf_layout(h, h->rgf_batch, h->rgf_meta_bytes);
  unsigned char* base = h->rgf_ws;
  const int64_t es = (int64_t)L.est;
  cplx* B0 = reinterpret_cast<cplx*>(base + L.blk);
  auto blk = [&](size_t k) { return B0 + k * b2; };
  const size_t wk = 2 * (size_t)ny;
  cplx* G0[2] = {blk(wk), blk(wk + 1)};
  cplx* GN[2] = {blk(wk + 2), blk(wk + 3)};
  cplx* D[2] = {blk(wk + 4), blk(wk + 5)};
  cplx* Wb = blk(wk + 6);
  cplx* Xb = blk(wk + 8);
  auto gops = reinterpret_cast<const findgb::GemmOp*>(base + L.meta + h->rgf_tab[0]);
  auto iops = reinterpret_cast<const findgb::InvOp*>(base + L.meta + h->rgf_tab[1]);
  auto zmap = reinterpret_cast<const int*>(base + L.meta + h->rgf_tab[2]);
  const int ntiles = ((nx + 63) / 64) * ((nx + 63) / 64);
  int* status = reinterpret_cast<int*>(base + L.stat);
  cplx* dE = reinterpret_cast<cplx*>(base + L.E);
  cplx* sig = reinterpret_cast<cplx*>(base + L.sig);
  cplx* SL = reinterpret_cast<cplx*>(base + L.SL);
  cplx* SR = reinterpret_cast<cplx*>(base + L.SR);
  const bool dG = device_accessible(G), dGl = device_accessible(Gl);
  cudaError_t e = cudaMemsetAsync(status, 0x7f, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  auto gemm = [&](int op, int nb) { findgb::launch_gemm(gops + op, zmap, ntiles, 1, nb, st, 0, 0, 0); };
  for (int e0 = 0; e0 < nE; e0 += batch) {
    const int nb = std::min(batch, nE - e0);
    e = cudaMemcpyAsync(dE, E + 2 * (int64_t)e0, nb * sizeof(cplx), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy copy");
    findgb::launch_lead_modes(dE, nb, reinterpret_cast<const double*>(base + L.eps),
                              reinterpret_cast<const double*>(base + L.tau), nx,
                              reinterpret_cast<cplx*>(base + L.modes), st);
    findgb::launch_lead_dense(reinterpret_cast<cplx*>(base + L.modes), reinterpret_cast<const double*>(base + L.phi),
                              nx, nb, sig, st);
    findgb::launch_rgf_lesser(sig, nx, fL, SL, nb, st);
    findgb::launch_rgf_lesser(sig, nx, fR, SR, nb, st);
    findgb::RgfSlice s;
    s.nx = nx; s.ny = ny; s.stencil = p.stencil;
    s.t = h->desc.t; s.tp = h->desc.tp; s.onsite0 = h->desc.onsite0;
    s.V = reinterpret_cast<const double*>(base + L.V);
    s.E = dE; s.sigL = sig; s.sigR = sig;
    cplx* oG = dG ? reinterpret_cast<cplx*>(G) + (int64_t)e0 * n : reinterpret_cast<cplx*>(base + L.G);
    cplx* oGl = dGl ? reinterpret_cast<cplx*>(Gl) + (int64_t)e0 * n : reinterpret_cast<cplx*>(base + L.Gl);
    // right-connected sweep
    for (int y = ny - 1; y >= 0; --y) {
      findgb::launch_rgf_block(s, y, y < ny - 1 ? blk(y + 1) : nullptr, es, blk(y), es, nb, st);
      findgb::launch_invert(iops + 2 * y, 1, nx, status, e0, nb, st);
    }
    // first column G_y0 and its share of diag G<
    for (int y = 0; y < ny; ++y) {
      if (y > 0) {
        findgb::launch_rgf_cprod(s, y == 1 ? blk(0) : G0[(y - 1) & 1], es, Wb, es, 1.0, 0, nb, st);
        gemm(2 * y, nb);
      }
      gemm(2 * y + 1, nb);
      findgb::launch_rgf_diag(s, Xb, y == 0 ? blk(0) : G0[y & 1], es, oGl + (int64_t)y * nx, n, 0, nullptr,
                              nullptr, nb, st);
    }
    // left-connected sweep
    for (int y = 0; y < ny; ++y) {
      findgb::launch_rgf_block(s, y, y > 0 ? blk((size_t)ny + y - 1) : nullptr, es, blk((size_t)ny + y), es, nb, st);
      findgb::launch_invert(iops + 2 * y + 1, 1, nx, status, e0, nb, st);
    }
    // backward: G_yy, G_{y,N-1}, diag G, the second share of diag G<
    const int ob = 2 * ny;
    const cplx* prevD = blk((size_t)ny + ny - 1);
    const cplx* prevGN = prevD;
    gemm(ob + 4 * (ny - 1) + 3, nb);
    findgb::launch_rgf_diag(s, Xb, prevGN, es, oGl + (int64_t)(ny - 1) * nx, n, 1, prevD,
                            oG + (int64_t)(ny - 1) * nx, nb, st);
    for (int y = ny - 2; y >= 0; --y) {
      findgb::launch_rgf_cprod(s, prevD, es, Wb, es, 1.0, 1, nb, st);  // W = C G_{y+1,y+1} C
      gemm(ob + 4 * y, nb);                                           // T = gL_y W
      gemm(ob + 4 * y + 1, nb);                                       // D_y = gL_y + T gL_y
      findgb::launch_rgf_cprod(s, prevGN, es, Wb, es, 1.0, 0, nb, st); // W = C G_{y+1,N-1}
      gemm(ob + 4 * y + 2, nb);                                       // GN_y = -gL_y W
      gemm(ob + 4 * y + 3, nb);                                       // X = GN_y S<_R
      findgb::launch_rgf_diag(s, Xb, GN[y & 1], es, oGl + (int64_t)y * nx, n, 1, D[y & 1],
                              oG + (int64_t)y * nx, nb, st);
      prevD = D[y & 1];
      prevGN = GN[y & 1];
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "RGF launch");
    if (!dG) {
      e = cudaMemcpyAsync(G + 2 * (int64_t)e0 * n, oG, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "diagG copy-out");
    }
    if (!dGl) {
      e = cudaMemcpyAsync(Gl + 2 * (int64_t)e0 * n, oGl, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "diagGl copy-out");
    }
  }
  int hs = 0x7f7f7f7f;
  e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "RGF solve");
  if (hs != 0x7f7f7f7f) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "exactly zero pivot at energy index %d", hs);
    return fail(h, FIND_ESINGULAR, buf);
  }
  h->err.clear();
  return FIND_OK;
}

}  // namespace

// ---------------------------------------------------------------- fixed device scratch
// Device memory of find_solve_diag_static, for callers that cannot allocate
// device memory.  It lives as long as the library stays loaded, on every
// device that uses it.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
constexpr int kMaxDevices = 128;
unsigned char* g_static_ptr[kMaxDevices] = {};

// Device address of the fixed scratch on `device`, which must be current.
// Looked up once per device; host code must never hand the symbol itself to a
// kernel (it is a host-side stand-in, not a device address).
cudaError_t static_scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_static_ptr[device];
  return cudaSuccess;
}

// The diag pass on the tables of `sv` (no profiling).
void run_level_static(find_handle* h, const StaticView& sv, const Level& lv,
                      const findgb::DevProblem& P, int e_base, int nb, cudaStream_t st, cplx* oG,
                      int sym_mask) {
  const Layout& L = sv.lay;
  auto meta = [&](size_t off) { return sv.base + L.meta + off; };
  auto pos = reinterpret_cast<const findgb::Pos*>(sv.base + L.pos);
  int* status = reinterpret_cast<int*>(sv.base + L.status);
  findgb::launch_assemble(reinterpret_cast<const findgb::AsmOp*>(meta(lv.asmops)),
                          reinterpret_cast<const int*>(meta(lv.row_op)), lv.nrows, pos, P, 0, nb, st);
  if (lv.leaf) {
    for (int c = 0; c < 4; ++c)
      findgb::launch_invert(reinterpret_cast<const findgb::InvOp*>(meta(lv.inv[c])), lv.ninv[c],
                            lv.inv_max[c], status, e_base, nb, st, 0, c & 1, c >> 1);
  } else {
    for (int c = 0; c < 2; ++c) {
      if (sv.ldl == 1)
        findgb::launch_ldl(reinterpret_cast<const findgb::InvOp*>(meta(lv.inv[c])), lv.ninv[c],
                           lv.inv_max[c], status, e_base, nb, st, 0, c);
      else
        findgb::launch_lu(reinterpret_cast<const findgb::InvOp*>(meta(lv.inv[c])), lv.ninv[c],
                          lv.inv_max[c], status, e_base, nb, st, 0, c);
    }
    for (int c = 0; c < 2; ++c)
      findgb::launch_trsm(reinterpret_cast<const findgb::TrsmOp*>(meta(lv.trsm)),
                          reinterpret_cast<const int*>(meta(lv.trsm_map[c])), lv.ntrsm[c], lv.rb,
                          lv.max_s, nb, st, c, 0, sv.ldl == 1 ? 0 : ff_factors(h, c), sv.ldl == 1);
  }
  for (int k = 0; k < lv.nstages; ++k) {
    const Stage& s = lv.st[k];
    auto ops = reinterpret_cast<const findgb::GemmOp*>(meta(s.ops));
    for (int c = 0; c < 6; ++c)
      findgb::launch_gemm(ops, reinterpret_cast<const int*>(meta(s.map[c])), s.nmap[c], c & 1, nb, st,
                          c >> 1, 0, sym_mask);
    for (const TcChunk& c : s.tc) {
      auto tops = reinterpret_cast<const findgb::TcOp*>(meta(c.ops));
      findgb::launch_tc_split(c.L, tops, reinterpret_cast<const int4*>(meta(c.sitems)), c.nsitems,
                              reinterpret_cast<const int4*>(meta(c.ritems)), c.nritems,
                              reinterpret_cast<const int4*>(meta(c.citems)), c.ncitems, nb, st);
      findgb::launch_tc_mma(c.L, tops, reinterpret_cast<const int*>(meta(c.tmap)), c.ntiles, status, nb, st);
    }
  }
  if (lv.leaf)
    findgb::launch_extract(reinterpret_cast<const findgb::ExtractOp*>(meta(lv.ext)), lv.nops,
                           reinterpret_cast<const findgb::LeafBond*>(sv.base + L.bonds), P, 0, 0, oG,
                           nullptr, nullptr, (int64_t)h->plan.nx * h->plan.ny, h->plan.n_bonds, nb, st);
}

int solve_static(find_handle* h, const double* E, int nE, const double* sigL, const double* sigR,
                 double* G, void* stream) {
  if (!h) return fail(nullptr, FIND_EINVAL, "null handle");
  if (nE < 0) return fail(h, FIND_EINVAL, "nE < 0");
  if (nE == 0) return FIND_OK;
  if (!E || !G) return fail(h, FIND_EINVAL, "E and diagG must not be NULL");
  DeviceGuard guard(h->desc.device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = static_scratch_address(h->desc.device, &base);
  if (e != cudaSuccess) return cuda_fail(h, e, "fixed scratch address");
  StaticView& sv = h->sview;
  const int ldl = (default_ldl(h) && !sigL && !sigR) ? 1 : 0;
  if (sv.base != base || sv.ldl != ldl) {
    // the largest energy batch that fits: the footprint is an affine
    // function of the batch (per-energy slabs plus fixed tables), taken from
    // two table builds and confirmed by a third
    int batch = 0;
    const double need1 = workspace_bytes(h, 1, false, nullptr, ldl);
    if (need1 <= (double)kStaticScratchBytes) {
      const double per = std::max(1.0, workspace_bytes(h, 2, false, nullptr, ldl) - need1);
      batch = std::max(1, std::min(64, 1 + (int)(((double)kStaticScratchBytes - need1) / per)));
      while (batch > 1 && workspace_bytes(h, batch, false, nullptr, ldl) > (double)kStaticScratchBytes)
        --batch;
    }
    if (batch == 0) {
      char buf[192];
      std::snprintf(buf, sizeof buf,
                    "this mesh needs %.1f MiB of device scratch for one energy; the fixed scratch of "
                    "find_solve_diag_static holds %.0f MiB",
                    need1 / 1048576.0, (double)kStaticScratchBytes / 1048576.0);
      return fail(h, FIND_EINVAL, buf);
    }
    Arena sizing;
    std::vector<Level> lv;
    int64_t se = 0;
    h->ldl_build = ldl != 0;
    Layout L0 = make_layout(h, batch, false, 0, 0);
    build_tables(h, nullptr, L0, batch, false, sizing, lv, se);
    Layout L = make_layout(h, batch, false, se, sizing.buf.size());
    Arena real;
    Bounds bc;
    bc.lo = base;
    bc.hi = base + L.meta;
    bc.s_lo = base + L.scratch;
    bc.s_hi = base + L.scratch + (size_t)se * batch * sizeof(cplx);
    bc.s_stride = se * (int64_t)sizeof(cplx);
    int map_err = 0;
    build_tables(h, base, L, batch, false, real, lv, se, &bc, &map_err);
    if (!bc.err.empty() || L.total > kStaticScratchBytes)
      return fail(h, FIND_EINVAL, "internal table check failed for the fixed scratch: " + bc.err);
    if (map_err) return fail(h, FIND_ECUDA, "tensor map encoding of the digit planes failed");
    sv.base = base;
    sv.ldl = ldl;
    sv.batch = batch;
    sv.lay = L;
    sv.levels = std::move(lv);
    sv.meta = std::move(real.buf);
  }
  const findgb::Plan& p = h->plan;
  const Layout& L = sv.lay;
  const int64_t n = (int64_t)p.nx * p.ny, nx = p.nx;
  // the array is shared by every handle: upload this handle's constants and
  // tables on each call, and clear the status word
  struct Up { size_t off; const void* src; size_t bytes; } ups[] = {
      {L.V, h->V.data(), h->V.size() * 8},
      {L.phi, h->phi.data(), h->phi.size() * 8},
      {L.eps, h->eps.data(), h->eps.size() * 8},
      {L.tau, h->tau.data(), h->tau.size() * 8},
      {L.pos, p.pos.data(), p.pos.size() * sizeof(findgb::Pos)},
      {L.bonds, p.bonds.data(), p.bonds.size() * sizeof(findgb::LeafBond)},
      {L.meta, sv.meta.data(), sv.meta.size()}};
  for (const Up& u : ups) {
    if (u.bytes == 0) continue;
    e = cudaMemcpyAsync(base + u.off, u.src, u.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "fixed scratch upload");
  }
  int* status = reinterpret_cast<int*>(base + L.status);
  e = cudaMemsetAsync(status, 0x7f, 2 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  const int kNoError = 0x7f7f7f7f;
  cplx* dE = reinterpret_cast<cplx*>(base + L.E);
  cplx* dsL = reinterpret_cast<cplx*>(base + L.sigL);
  cplx* dsR = reinterpret_cast<cplx*>(base + L.sigR);
  cplx* dmodes = reinterpret_cast<cplx*>(base + L.modes);
  const bool dG = device_accessible(G);
  for (int e0 = 0; e0 < nE; e0 += sv.batch) {
    const int nb = std::min(sv.batch, nE - e0);
    e = cudaMemcpyAsync(dE, E + 2 * (int64_t)e0, nb * sizeof(cplx), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "energy copy");
    const cplx* useL = dsL;
    const cplx* useR = dsR;
    if (!sigL || !sigR) {
      cplx* dst = !sigL ? dsL : dsR;
      findgb::launch_lead_modes(dE, nb, reinterpret_cast<const double*>(base + L.eps),
                                reinterpret_cast<const double*>(base + L.tau), (int)nx, dmodes, st);
      findgb::launch_lead_dense(dmodes, reinterpret_cast<const double*>(base + L.phi), (int)nx, nb, dst, st);
      if (!sigL && !sigR) useR = dsL;
    }
    if (sigL) {
      e = cudaMemcpyAsync(dsL, sigL + 2 * (int64_t)e0 * nx * nx, nb * nx * nx * sizeof(cplx),
                          cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "sigmaL copy");
    }
    if (sigR) {
      e = cudaMemcpyAsync(dsR, sigR + 2 * (int64_t)e0 * nx * nx, nb * nx * nx * sizeof(cplx),
                          cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "sigmaR copy");
    }
    findgb::DevProblem P;
    P.nx = p.nx; P.ny = p.ny; P.stencil = p.stencil;
    P.t = h->desc.t; P.tp = h->desc.tp; P.onsite0 = h->desc.onsite0;
    P.V = reinterpret_cast<const double*>(base + L.V);
    P.E = dE; P.sigL = useL; P.sigR = useR;
    P.fL = 0.0; P.fR = 0.0;
    P.dles = nullptr; P.dles_estride = 0;
    cplx* oG = dG ? reinterpret_cast<cplx*>(G) + (int64_t)e0 * n : reinterpret_cast<cplx*>(base + L.oG);
    const int sym_mask = sym_updates(h, sigL, sigR);
    for (const Level& lv : sv.levels) run_level_static(h, sv, lv, P, e0, nb, st, oG, sym_mask);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "kernel launch");
    if (!dG) {
      e = cudaMemcpyAsync(G + 2 * (int64_t)e0 * n, oG, nb * n * sizeof(cplx), cudaMemcpyDefault, st);
      if (e != cudaSuccess) return cuda_fail(h, e, "diagG copy-out");
    }
  }
  int hs2[2] = {kNoError, kNoError};
  e = cudaMemcpyAsync(hs2, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve");
  if (hs2[1] != kNoError) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "a bounded wait of the tensor-core product ran out (role %d)", hs2[1]);
    return fail(h, FIND_ETIMEOUT, buf);
  }
  const int hs = hs2[0];
  if (hs != kNoError) {
    char buf[128];
    std::snprintf(buf, sizeof buf, "exactly zero pivot at energy index %d", hs);
    return fail(h, FIND_ESINGULAR, buf);
  }
  h->err.clear();
  return FIND_OK;
}

}  // namespace

extern "C" {

int find_create(const find_desc* d, find_handle** out) {
  if (!d || !out) return fail(nullptr, FIND_EINVAL, "null descriptor or output");
  *out = nullptr;
  if (d->precision != FIND_FP64 && d->precision != FIND_MIXED && d->precision != FIND_MIXED_FF)
    return fail(nullptr, FIND_EINVAL, "precision must be FIND_FP64, FIND_MIXED or FIND_MIXED_FF");
  if (d->stencil != 5 && d->stencil != 9) return fail(nullptr, FIND_EINVAL, "stencil must be 5 or 9");
  if (d->max_batch < 0) return fail(nullptr, FIND_EINVAL, "max_batch < 0");
  if (d->gemm_small_max < 0) return fail(nullptr, FIND_EINVAL, "gemm_small_max < 0");
  if (d->tc_slices < 0 || d->tc_slices > 12 || d->tc_slices_mixed < 0 || d->tc_slices_mixed > 12 ||
      d->tc_min < 0)
    return fail(nullptr, FIND_EINVAL, "tc_slices and tc_slices_mixed must be in [0, 12], tc_min >= 0");
  if (d->flags & ~(FIND_FLAG_FULL_U | FIND_FLAG_SYM_U | FIND_FLAG_GRAPH | FIND_FLAG_NO_TC | FIND_FLAG_LU |
                   FIND_FLAG_LDL))
    return fail(nullptr, FIND_EINVAL, "unknown bit in flags");
  if (d->energy_group < 0 || d->sigma_c64_depth < 0)
    return fail(nullptr, FIND_EINVAL, "energy_group and sigma_c64_depth must be >= 0");
  find_handle* h = new (std::nothrow) find_handle();
  if (!h) return fail(nullptr, FIND_ENOMEM, "host allocation");
  h->desc = *d;
  h->desc.onsite_V = nullptr;
  if (h->desc.leaf <= 0) h->desc.leaf = 8;
  std::string err;
  if (findgb::build_plan(d->nx, d->ny, d->stencil, h->desc.leaf, h->plan, err) != 0) {
    delete h;
    return fail(nullptr, FIND_EINVAL, err);
  }
  if (std::max(h->plan.max_s, h->plan.max_kn) > findgb::kMaxInvert) {
    delete h;
    return fail(nullptr, FIND_EINVAL, "a private-inner or bordered leaf set exceeds 2048 nodes");
  }
  const size_t n = (size_t)d->nx * d->ny;
  h->V.assign(n, 0.0);
  if (d->onsite_V) {
    if (device_accessible(d->onsite_V)) {
      cudaError_t e = cudaMemcpy(h->V.data(), d->onsite_V, n * 8, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        delete h;
        return fail(nullptr, FIND_ECUDA, std::string("onsite_V copy: ") + cudaGetErrorString(e));
      }
    } else {
      std::memcpy(h->V.data(), d->onsite_V, n * 8);
    }
  }
  // transverse sine modes of the leads: phi[x][m], eps_m, tau_m
  const int nx = d->nx;
  h->phi.resize((size_t)nx * nx);
  h->eps.resize(nx);
  h->tau.resize(nx);
  const double pi = 3.14159265358979323846;
  for (int m = 1; m <= nx; ++m) {
    double th = m * pi / (nx + 1);
    h->eps[m - 1] = d->onsite0 - 2.0 * d->t * std::cos(th);
    h->tau[m - 1] = (d->stencil == 9) ? -d->t - 2.0 * d->tp * std::cos(th) : -d->t;
    for (int x = 0; x < nx; ++x)
      h->phi[(size_t)x * nx + (m - 1)] = std::sqrt(2.0 / (nx + 1)) * std::sin(m * (x + 1) * pi / (nx + 1));
  }
  *out = h;
  return FIND_OK;
}

int find_plan_info(const find_handle* h, find_plan_stats* o) {
  if (!h || !o) return FIND_EINVAL;
  const findgb::Plan& p = h->plan;
  o->n_clusters = (int)p.cl.size();
  o->n_leaves = p.n_leaves;
  o->n_up_levels = (int)p.up_levels.size();
  o->n_down_levels = (int)p.dn_levels.size();
  o->max_s = p.max_s;
  o->max_b = p.max_b;
  o->max_kn = p.max_kn;
  o->n_bonds = p.n_bonds;
  o->flops_diag = p.flops_diag;
  o->flops_lesser = p.flops_lesser;
  o->ur_bytes = 2.0 * (double)p.mat_elems * sizeof(cplx);
  find_handle* hh = const_cast<find_handle*>(h);
  o->scratch_bytes = workspace_bytes(hh, 2, true) - workspace_bytes(hh, 1, true) - o->ur_bytes -
                     (double)(3 * (size_t)p.nx * p.ny * 16 + 2 * (size_t)p.nx * p.nx * 16);
  return FIND_OK;
}

int find_workspace_bytes(const find_handle* h, int batch, int lesser, double* bytes) {
  if (!h || !bytes || batch < 1) return FIND_EINVAL;
  find_handle* hh = const_cast<find_handle*>(h);
  std::string err;
  *bytes = workspace_bytes(hh, batch, lesser != 0, &err);
  if (!err.empty()) return fail(hh, FIND_EINVAL, "internal table check failed: " + err);
  return FIND_OK;
}

int find_solve_diag(find_handle* h, const double* E, int nE, const double* sigmaL,
                    const double* sigmaR, double* diagG, void* stream) {
  return solve(h, E, nE, sigmaL, sigmaR, 0.0, 0.0, nullptr, 0, diagG, nullptr, nullptr, stream, false);
}

int find_rgf_solve_lesser(find_handle* h, const double* E, int nE, double fL, double fR,
                          double* diagG, double* diagGl, void* stream) {
  return rgf_solve(h, E, nE, fL, fR, diagG, diagGl, stream);
}

int find_solve_diag_static(find_handle* h, const double* E, int nE, const double* sigmaL,
                           const double* sigmaR, double* diagG, void* stream) {
  return solve_static(h, E, nE, sigmaL, sigmaR, diagG, stream);
}

int find_solve_lesser(find_handle* h, const double* E, int nE, const double* sigmaL,
                      const double* sigmaR, double fL, double fR, const double* sigma_lesser_diag,
                      int diag_per_energy, double* diagG, double* diagGl, double* bond_current,
                      void* stream) {
  return solve(h, E, nE, sigmaL, sigmaR, fL, fR, sigma_lesser_diag, diag_per_energy, diagG, diagGl,
               bond_current, stream, true);
}

int find_profile(find_handle* h, int enable) {
  if (!h) return FIND_EINVAL;
  DeviceGuard guard(h->desc.device);
  for (auto& p : h->pending) {
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->pending.clear();
  if (enable) {
    std::memset(h->stats, 0, sizeof(h->stats));
    for (int k = 0; k < kClasses; ++k)
      std::snprintf(h->stats[k].name, sizeof h->stats[k].name, "%s", kClassNames[k]);
  }
  h->prof = enable != 0;
  return FIND_OK;
}

int find_profile_read(find_handle* h, find_kernel_stat* out, int max, int* count) {
  if (!h || (!out && max > 0)) return FIND_EINVAL;
  DeviceGuard guard(h->desc.device);
  for (auto& p : h->pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(p.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
    if (e != cudaSuccess) return cuda_fail(h, e, "profile events");
    find_kernel_stat& s = h->stats[p.cls];
    s.launches += 1;
    s.ms += ms;
    s.flops += p.flops;
    s.bytes += p.bytes;
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->pending.clear();
  for (int k = 0; k < kClasses && k < max; ++k) out[k] = h->stats[k];
  if (count) *count = kClasses;
  return FIND_OK;
}

int find_destroy(find_handle* h) {
  if (!h) return FIND_OK;
  {
    DeviceGuard guard(h->desc.device);
    release(h);
    for (auto& p : h->pending) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (auto e : h->ev_free) cudaEventDestroy(e);
    for (auto e : h->gevents) cudaEventDestroy(e);
    for (auto q : h->gstreams) cudaStreamDestroy(q);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  }
  delete h;
  return FIND_OK;
}

const char* find_last_error(const find_handle* h) {
  return h ? h->err.c_str() : g_create_error.c_str();
}

}  // extern "C"
