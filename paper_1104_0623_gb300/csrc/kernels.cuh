// Descriptors shared by the host runtime and the CUDA kernels of the FIND
// passes, and the launch wrappers.  All complex data are interleaved double
// pairs (double2: x = re, y = im).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "plan.hpp"  // Pos, LeafBond

namespace findgb {

typedef double2 cplx;

// Per-call constants of the mesh problem A = E I - H - Sigma_L - Sigma_R.
struct DevProblem {
  int nx, ny, stencil;
  double t, tp, onsite0;
  const double* V;         // n onsite disorder values
  const cplx* E;           // energies of the current pass
  const cplx* sigL;        // [e][nx][nx]
  const cplx* sigR;        // [e][nx][nx]
  double fL, fR;
  const cplx* dles;        // node-diagonal Sigma< or nullptr
  int64_t dles_estride;    // 0 when shared by all energies
};

// Assembly of one op: M (and Sigma_M) over n positions, one CTA per row.
struct AsmOp {
  int n, row0;
  int64_t pos;
  const cplx* u1; const cplx* r1; int d1;  // source 1 (energy 0), stride d1*d1; r1 null: R = 0
  const cplx* u2; const cplx* r2; int d2;  // source 2
  cplx* M;                                 // energy 0; S_M = M + n*n
  int64_t estride;                         // per-energy stride of the op scratch
  int sig;  // lesser passes: 1 writes Sigma_M; 0: Sigma_M is zero and nothing reads it
};

// In-place Gauss-Jordan inversion of the leading s x s block of M (ld); with
// piv != nullptr, an in-place LU factorisation P M = L U of that block
// instead (row interchanges in piv, LAPACK order).
struct InvOp {
  cplx* M;
  int64_t estride;
  int ld, s;
  int* piv;
  int64_t piv_estride;
  cplx* dv;             // LDL^T only: D (2 s entries: diagonal, then the
                        // sub-diagonal of the 2x2 blocks), stride estride
};

// L = M(B,S) M(S,S)^{-1} from the LU factors of M(S,S): rows r0..r0+rb of
// M(B,S) per CTA; Y U = M(B,S), Z L = Y, L = Z P.
//
// LDL^T factors (k_ldl): P M(S,S) P^T = T D T^T.  Then L = M(B,S) P^T T^-T
// D^-1 T^-1 P by the same two sweeps: the rows are first permuted by P^T,
// the forward sweep with T^T gives W^T (rows of M(B,S) P^T T^-T), which is
// stored together with W^T D^-1 (for U = M(B,B) - (W^T D^-1) W, the
// symmetric form of Eq. 2); then the backward sweep with T and P.
struct TrsmOp {
  const cplx* M;        // energy 0; M(S,S) holds the factors, M(B,S) the rows
  int64_t estride;
  int ld, s, b;
  const int* piv;       // LDL^T: piv[s] interchanges, then kind[s] block flags
  int64_t piv_estride;
  cplx* L;              // b x s, leading dimension s
  int64_t l_estride;    // also the stride of dv, Wt and Yd
  int tile0;            // first row-block of this op in the launch
  const cplx* dv;       // LDL^T: D as in InvOp::dv
  cplx* Wt;             // LDL^T: W^T, b x s
  cplx* Yd;             // LDL^T: W^T D^-1, b x s
};

// D = beta * C + alpha * A op(B) + alpha2 * A2 op(B2); op(B) = B (opb 0),
// B^H (opb 1, B stored n x k) or B^T (opb 2, B stored n x k).  Every operand is row-major with its leading
// dimension and a per-energy stride.
struct GemmOp {
  int m, n, k, k2;
  const cplx* A; int lda; int64_t sa;
  const cplx* B; int ldb; int64_t sb; int opb;
  const cplx* A2; int lda2; int64_t sa2;
  const cplx* B2; int ldb2; int64_t sb2; int opb2;
  const cplx* C; int ldc; int64_t sc;
  cplx* D; int ldd; int64_t sd;
  double alpha, alpha2, beta;
  int tile0, tiles_n;
  int sym;  // 1: D is complex symmetric (m == n) when the problem is; the
            // launch's sym_mask decides whether only the upper triangle is
            // computed and mirrored
};

struct ExtractOp {
  const cplx* K;       // inverted bordered system G_K (energy 0), n x n
  const cplx* Q;       // rows C of G<_K (energy 0), c x n
  int64_t estride;
  int n, nb, c;
  int x0, y0, wx;
  int64_t bond;
  int nbond;
};

// ---- launch wrappers (kernels.cu)
void launch_lead_modes(const cplx* E, int nE, const double* eps, const double* tau, int nx,
                       cplx* sig_modes, cudaStream_t st);
void launch_lead_dense(const cplx* sig_modes, const double* phi, int nx, int nE, cplx* out,
                       cudaStream_t st);
// Every launch covers energies e_off .. e_off + nE - 1 of the current pass
// (grid.y = nE); independent energy groups can run on separate streams.
void launch_assemble(const AsmOp* ops, const int* row_op, int nrows, const Pos* pos,
                     const DevProblem& P, int lesser, int nE, cudaStream_t st, int e_off = 0);
// Blocks of at most this many rows are factorised (LU, LDL^T) by thread
// blocks of 128 threads (256 up to twice that, 512 above): per-step barriers
// and pivot searches then span fewer warps, and more blocks share an SM.
constexpr int kSmallBlock = 128;
// df = 1: float-float arithmetic; in_smem = 1: the block is held in shared
// memory (every op of the launch must have s <= invert_smem_max())
void launch_invert(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
                   cudaStream_t st, int e_off = 0, int df = 0, int in_smem = 0);
int invert_smem_max();
void launch_lu(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
               cudaStream_t st, int e_off = 0, int df = 0);
// Bunch-Kaufman LDL^T of the complex symmetric M(S,S) (Sec. 4.2); df = 1:
// float-float arithmetic (the factors still leave as complex128)
void launch_ldl(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
                cudaStream_t st, int e_off = 0, int df = 0);
// df = 1: the row block is carried in float-float arithmetic; ff_factors = 1:
// the LU factors of M(S,S) are float-float words (the float-float LU leaves
// them so), else complex128
void launch_trsm(const TrsmOp* ops, const int* tile_op, int ntiles, int rb, int max_s, int nE,
                 cudaStream_t st, int df = 0, int e_off = 0, int ff_factors = 0, int ldl = 0);
int trsm_rows_per_block(int max_s);
// fp32 = 1: complex64 arithmetic on complex128 operands (mixed path);
// fp32 = 2: float-float arithmetic (about 48 significant bits)
// sym_mask bit 0: ops with sym == 1 compute the upper triangle and mirror it
void launch_gemm(const GemmOp* ops, const int* tile_op, int ntiles, int big, int nE,
                 cudaStream_t st, int fp32 = 0, int e_off = 0, int sym_mask = 0);
void launch_extract(const ExtractOp* ops, int nops, const LeafBond* bonds, const DevProblem& P,
                    int lesser, int want_bonds, cplx* diagG, cplx* diagGl, double* J,
                    int64_t n_nodes, int64_t n_bonds, int nE, cudaStream_t st, int e_off = 0);

constexpr int kMaxInvert = 2048;  // largest block the in-CTA inversion accepts

// ---- recursive Green's function baseline (rgf.cu)
struct RgfSlice {
  int nx, ny, stencil;
  double t, tp, onsite0;
  const double* V;      // nx*ny onsite disorder
  const cplx* E;        // energies of the pass
  const cplx* sigL;     // [e][nx][nx]
  const cplx* sigR;
};
// M = A_yy - C X C (X may be nullptr), per energy (strides in complex entries)
void launch_rgf_block(const RgfSlice& s, int y, const cplx* X, int64_t xstride, cplx* M, int64_t mstride,
                      int nE, cudaStream_t st);
// W = sign C X, or C X C with sandwich = 1
void launch_rgf_cprod(const RgfSlice& s, const cplx* X, int64_t xstride, cplx* W, int64_t wstride,
                      double sign, int sandwich, int nE, cudaStream_t st);
// out[x] (+)= (P Q^H)_xx; diagG[x] = diag_src[x][x] when diag_src is given
void launch_rgf_diag(const RgfSlice& s, const cplx* P, const cplx* Q, int64_t stride, cplx* out,
                     int64_t ostride, int accumulate, const cplx* diag_src, cplx* diagG, int nE,
                     cudaStream_t st);
// out = -f (sig - sig^H) per energy
void launch_rgf_lesser(const cplx* sig, int nx, double f, cplx* out, int nE, cudaStream_t st);

// ---- tensor-core products (tc_gemm.cu): D = beta C + a1 A1 op(B1) + a2 A2 op(B2)
// computed from bf16 digit planes of the operands (see tc_gemm.cu).
struct TcOp {
  int m, n;              // output rows, columns
  int k1, k2;            // inner dimensions of the two products (k2 = 0: none)
  int k1p, kp;           // k1 padded to 64 (offset of the second product), total padded K
  int mt, tiles_n;       // 128-row and 128-column tiles
  int tile0;             // first tile of this op in the launch
  int nsl, nexact;       // digit planes per operand; exactly accumulated diagonals
  int arow, brow;        // first plane row of A / op(B) in the slab (per energy)
  int ascale, bscale;    // first exponent of the rows of A / columns of op(B)
  const cplx* A1; int lda1; int64_t sa1; int neg1;
  const cplx* B1; int ldb1; int64_t sb1; int opb1;
  const cplx* A2; int lda2; int64_t sa2; int neg2;
  const cplx* B2; int ldb2; int64_t sb2; int opb2;
  const cplx* C; int ldc; int64_t sc; double beta;
  cplx* D; int ldd; int64_t sd;
};

// Digit planes and exponents of one launch, energy 0; energy e at + e * estride.
// A plane (s, part) of op o holds rows o.arow + (2 s + part) * 128 o.mt ...,
// each `pitch` bf16 long (K-contiguous).
struct TcSlab {
  unsigned short* a;
  unsigned short* b;
  int64_t pitch;          // bf16 per plane row
  int64_t plane_estride;  // bf16 between energies
  int* scale;
  int64_t scale_estride;  // ints between energies
};

struct TcLaunch {
  TcSlab slab;
  int scale_ints;          // exponents per energy
  alignas(64) unsigned char mapA[128];  // CUtensorMap of the A planes (3D: K, row, energy)
  alignas(64) unsigned char mapB[128];
};

// Encodes the 3D tensor map (K pitch_elems, rows, energies; energy stride in
// bytes) of a bf16 plane slab with 64 x 128 boxes and the 128-byte swizzle.
// Returns 0 on success.
int tc_encode_map(void* map_out, const void* base, int64_t pitch_elems, int64_t rows,
                  int64_t energies, int64_t estride_bytes);
int tc_tile_m();
int tc_tile_n();
int tc_tile_k();
int tc_smem_bytes();

// Host tables of one tensor-core launch: ops (with their plane rows, exponent
// offsets and tiles assigned by tc_add_op), work items and the tile -> op map.
struct TcBuild {
  std::vector<TcOp> ops;
  std::vector<int4> scale_items, row_items, col_items;
  std::vector<int> tile_op;
  int64_t rowsA = 0, rowsB = 0, pitch = 0;
  int scale_ints = 0;
};
// Adds an op given m, n, k1, k2, nsl, nexact and its operands.
void tc_add_op(TcBuild& b, TcOp op);
// Bytes per energy of the launch's planes and exponents, and their offsets.
int64_t tc_slab_bytes(const TcBuild& b, int64_t* offA, int64_t* offB, int64_t* offS);
// Slab bytes one op alone needs (planes and exponents, per energy).
int64_t tc_op_slab_bytes(int m, int n, int k1, int k2, int nsl);
// The two halves of launch_tc_gemm: exponents and digit planes; products.
void launch_tc_split(const TcLaunch& L, const TcOp* ops, const int4* scale_items, int nscale,
                     const int4* row_items, int nrow, const int4* col_items, int ncol, int nE,
                     cudaStream_t st, int e_off = 0);
void launch_tc_mma(const TcLaunch& L, const TcOp* ops, const int* tile_op, int ntiles, int* status,
                   int nE, cudaStream_t st, int e_off = 0);
// Splits the operands of every op into digit planes and runs the products.
// items (one per CTA): scale (op, kind | part << 4, i0, k0), rows (op, side,
// r0), cols (op, part, j0, k0); status[1] records a bounded wait that ran out.
void launch_tc_gemm(const TcLaunch& L, const TcOp* ops, const int4* scale_items, int nscale,
                    const int4* row_items, int nrow, const int4* col_items, int ncol,
                    const int* tile_op, int ntiles, int* status, int nE, cudaStream_t st,
                    int e_off = 0);

}  // namespace findgb
