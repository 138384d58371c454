/*
 * find.h -- C ABI of the GB300 FIND selected-inversion library.
 *
 * FIND (Fast Inverse using Nested Dissection; Li & Darve, "Extension and
 * optimization of the FIND algorithm") computes selected entries of
 *     G  = A^{-1}                     (Sec. 2)
 *     G< = A^{-1} Sigma< A^{-H}        (Sec. 3.1, Eq. 5)
 * for the sparse matrix of a 2D Nx x Ny tight-binding mesh
 *     A = E I - H - Sigma_L - Sigma_R  (Sec. 1; E is complex, eta included)
 * by an upward pass (Procedure updateBoundaryNodes), a downward pass
 * (Procedure updateAdjacentNodes) and per-leaf extraction (Procedure
 * computeG<, Eqs. 8-10), all run as CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *   - node n = y * nx + x; x in [0, nx) is transverse, y in [0, ny) is the
 *     transport direction; the leads attach to the columns y = 0 (left) and
 *     y = ny - 1 (right), nx nodes each.
 *   - H: onsite0 + V_n on the diagonal, -t to the 4 nearest neighbours,
 *     -tp to the 4 diagonal neighbours (stencil 9 only).
 *   - complex numbers are interleaved (re, im) pairs of double; "k complex"
 *     below means 2k doubles.
 *   - array pointers may be HOST or DEVICE memory; the library asks the CUDA
 *     runtime which one it is.  Host inputs are copied to the device on the
 *     given stream and host outputs are copied back.  A solve enqueues all
 *     of its work on `stream` and returns once the stream has completed it
 *     (it reads back the device status word of singular pivots), so every
 *     output is ready when the call returns.
 *   - one handle serves one host thread at a time; handles are independent.
 *   - ownership: the caller owns every array it passes; the handle owns the
 *     plan, the index tables and the resident U/R workspace.
 *   - errors: every call returns a FIND_* status; no partial outputs are
 *     promised on error; find_last_error() holds a message for the handle's
 *     last failing call.  Nothing aborts the process.
 */
#ifndef FIND_GB300_H
#define FIND_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FIND_OK = 0,
  FIND_EINVAL = 1,     /* bad argument: sizes, stencil, NULL where required */
  FIND_ENOMEM = 2,     /* device or host allocation failed                  */
  FIND_ESINGULAR = 3,  /* an exactly zero pivot was met (energy in message) */
  FIND_ETIMEOUT = 4,   /* a bounded device wait ran out                     */
  FIND_ECUDA = 5       /* any other CUDA runtime error                      */
};

/* FIND_FP64: every step in FP64.
 * FIND_MIXED: below the top fp64_top_levels tree levels, the Schur update U
 * (Eq. 2), the triangular solves for L (Eq. 13), the Sigma update (Eq. 7:
 * T = L Sigma(S,S) - Sigma(B,S), R = Sigma(B,B) - L Sigma(S,B) + T L^H) and
 * the leaf products G_K Sigma_K G_K^H run in float-float arithmetic (pairs of
 * floats, about 48 significant bits, on the FP32 pipes, which GB300 runs
 * about 70 times faster than FP64); the pivoted LU, the leaf inversion and
 * every step of the top levels stay FP64.  Operands and results stay
 * complex128 in memory.  Measured on the 256x1024 9-point mesh at 8 grid
 * energies: diag G and diag G< within 4.3e-8 of the exact values (FP64:
 * within 4e-10, and within a factor 5 of a plain FP64 FIND's own error).
 * FIND_MIXED_FF: as FIND_MIXED, and below the top levels the pivoted LU and
 * the leaf inversion run in float-float too.
 * Complex64 arithmetic is available for the Sigma update from a chosen tree
 * depth down (find_desc.sigma_c64_depth); it is faster, but on the 256x1024
 * mesh it left diag G< 4e-5 from the oracle (complex64 in the U update: up to
 * 2.5e-3 on a 64x128 mesh, so U never uses it). */
enum { FIND_FP64 = 0, FIND_MIXED = 1, FIND_MIXED_FF = 2 };

typedef struct find_handle find_handle;

typedef struct {
  int nx, ny;               /* mesh size, nx >= 1, ny >= 2                     */
  int stencil;              /* 5 or 9                                          */
  double t, tp;             /* nearest and diagonal hopping (tp used if 9)     */
  const double* onsite_V;   /* nx*ny doubles (host or device), copied at
                               find_create; NULL means V = 0                   */
  double onsite0;           /* clean onsite energy (4t, or 4t + 4tp for 9)     */
  int leaf;                 /* leaf clusters have both sides <= leaf; 0 = 8    */
  int precision;            /* FIND_FP64, FIND_MIXED or FIND_MIXED_FF          */
  int device;               /* CUDA device ordinal                             */
  int max_batch;            /* energies solved together; 0 = chosen from free
                               device memory                                   */
  int fp64_top_levels;      /* FIND_MIXED: tree depths 1..fp64_top_levels (the
                               root's children are depth 1) stay FP64; < 0
                               means the default 2                             */
  int energy_group;         /* energies per concurrent group within a pass
                               (groups run on their own streams, up to 4);
                               0 = 8                                           */
  int invert_smem;          /* bordered leaf systems up to this size are
                               inverted in shared memory (at most 112);
                               <= 0 = never (the default: measured slower)     */
  int sigma_c64_depth;      /* FIND_MIXED / _FF: the Sigma update of tree depths
                               >= this one (and > fp64_top_levels) runs in
                               complex64 instead of float-float; 0 = never     */
  int flags;                /* FIND_FLAG_* bits                                */
  int gemm_small_max;       /* a Schur-update or leaf product whose larger
                               output side is at most this runs on 32x32
                               tiles, a larger one on 64x64 tiles (a tuning
                               knob; results do not depend on it); 0 = per
                               product: 64x64 unless that pads more area than
                               the 32x32 tiling, by more than 20 % for
                               float-float and complex64, at all for FP64      */
  int tc_slices;            /* products that must match FP64 (every product of
                               FIND_FP64, the top levels of the mixed paths):
                               0 = FP64 on the CUDA cores (the default); 1..12
                               = on the tensor cores with this many digit
                               planes per operand (10 or more to match an FP64
                               product on operands of wide dynamic range)      */
  int tc_slices_mixed;      /* digit planes of the products the mixed paths run
                               below their top levels: 0 = 9 (about 2^-53
                               relative to the largest entries of the row of A
                               and the column of op(B)); at most 12            */
  int tc_min;               /* a product runs on the tensor cores when its
                               rows, columns and inner dimension are all at
                               least this (and its padding to the 128 x 128 x
                               64 tiles wastes little enough); 0 = 32          */
} find_desc;

/* find_desc.flags.  With the closed-form leads A = A^T, so every U is complex
   symmetric (Property 1) and its update can be computed on one triangle and
   mirrored.  That halves the U products but carries a larger rounding error:
   at 256x1024 the mirrored FP64 results were 3-10 times further from the
   exact values than with both triangles computed.  Default: both triangles on
   FIND_FP64, one triangle on the mixed paths (whose float-float rounding
   dominates).
     FIND_FLAG_FULL_U  both triangles on every path
     FIND_FLAG_SYM_U   one triangle on FIND_FP64 too (ignored with FULL_U)  */
enum { FIND_FLAG_FULL_U = 1, FIND_FLAG_SYM_U = 2, FIND_FLAG_GRAPH = 4, FIND_FLAG_NO_TC = 8,
       FIND_FLAG_LU = 16, FIND_FLAG_LDL = 32 };
/* Symmetric elimination (Sec. 4.2).  With the closed-form leads A = A^T, and
   FIND_FP64 eliminates every private inner set by LDL^T: M(S,S) is factored
   as P M(S,S) P^T = T D T^T with the diagonal pivoting of Bunch and Kaufman
   (1x1 and 2x2 blocks), W = T^-1 P M(S,B), and U = M(B,B) - W^T D^-1 W (Eq. 2
   in symmetric form); L = M(B,S) M(S,S)^-1 for Eq. 7 comes from the same
   factors.  Against the exact values on the 256x1024 mesh this form is tens
   to hundreds of times more accurate than the LU form at the energies where
   A is worst conditioned, and the factorisation takes half the LU's flops.
   A call that passes Sigma_L or Sigma_R (not known to be symmetric) uses the
   LU; switching between the two reallocates the workspace.  FIND_FLAG_LU
   keeps the LU elimination for every call.  The mixed paths (bar 1e-5) take
   the LU unless FIND_FLAG_LDL asks for the symmetric form, which makes them
   about 20 times more accurate at the worst energy but, on the 256x1024
   mesh, 26 % slower: their float-float LU is blocked in panels, the
   Bunch-Kaufman factorisation is not.  With FIND_FLAG_LDL the factorisation
   runs in the arithmetic of the path's LU (float-float below the top levels
   on FIND_MIXED_FF) and the solves in float-float.  FIND_FLAG_LU wins when
   both are set. */
/* Tensor-core products.  The Schur-update products (Eq. 2, Eq. 7) and the
   leaf products G_K Sigma_K G_K^H run by default on the bf16 tensor cores
   (tcgen05) through an error-free digit-plane split of the complex128
   operands (Ozaki et al. 2012): each row of A and each column of op(B) is
   scaled by a power of two and cut into signed base-64 digits; the digit
   products of one weight are accumulated exactly in FP32 tensor memory and
   summed as exact integers.  The error of a product entry is relative to the
   largest entries of its row of A and column of op(B) (about 2^-(6 planes)),
   not to the entries it sums, so operands whose rows decay over many decades
   (Green's-function blocks at energies near an inner resonance) need more
   planes than their FP64 precision suggests: on the 256x1024 mesh 9 planes
   left the FP64 path 200 times less accurate than FP64 products at the worst
   energy, so FP64 products stay on the CUDA cores unless tc_slices asks
   otherwise, while the mixed paths (bar 1e-5) take 9 planes.
   FIND_FLAG_NO_TC keeps every product on the CUDA-core kernels (FP64 or
   float-float). */
/* FIND_FLAG_GRAPH: find_solve_diag / find_solve_lesser capture the device work
   of a pass (closed-form lead Sigma and every level's launches, over all
   energy-group streams) into a CUDA graph the first time a call signature is
   seen -- the number of energies in the pass, its offset in the call, the
   outputs asked for, which of Sigma_L, Sigma_R and the node-diagonal Sigma<
   are given, fL, fR -- and replay it with cudaGraphLaunch afterwards (up to 8
   signatures per handle, least recently used dropped).  Energies and the
   optional inputs are copied in, and outputs copied out, outside the graph,
   so each call may pass new values and new buffers.  Results are bitwise
   the same as without the flag.  find_profile does not time replayed
   passes.  Reallocating the workspace (a larger batch) drops the graphs. */

/* Host-side facts of the plan (no GPU needed). */
typedef struct {
  int n_clusters;           /* basic clusters in the tree (root included)     */
  int n_leaves;
  int n_up_levels;          /* upward groups (by height)                       */
  int n_down_levels;        /* downward groups (by depth)                      */
  int max_s, max_b;         /* largest private-inner and boundary set          */
  int max_kn;               /* largest bordered leaf system |Bbar u C|         */
  int n_bonds;              /* bond-current outputs per energy                 */
  double flops_diag;        /* algorithmic real flops per energy, diag(G)     */
  double flops_lesser;      /* algorithmic real flops per energy, diag(G),
                               diag(G<) and bond currents                      */
  double ur_bytes;          /* resident U and R bytes per energy               */
  double scratch_bytes;     /* largest per-level scratch bytes per energy      */
} find_plan_stats;

/*
 * Build the nested-dissection tree (Sec. 2.1: bisect the longer side, ties
 * split y, first half floor(len/2)), the boundary sets B_C = {i in C with a
 * neighbour outside C}, the complement sets B_Cbar, the private inner sets
 * S_C = (B_C1 u B_C2) \ B_C, and the gather tables of every merge.
 * Touches no GPU; device memory is allocated by the first solve.
 * Returns FIND_EINVAL for nx < 1, ny < 2, a stencil other than 5 or 9, or a
 * set larger than the kernels support (2048).
 */
int find_create(const find_desc* desc, find_handle** out);

/* Plan facts; valid on any machine. */
int find_plan_info(const find_handle* h, find_plan_stats* out);

/* Bytes of device workspace a solve with `batch` energies per pass uses. */
int find_workspace_bytes(const find_handle* h, int batch, int lesser, double* bytes);

/*
 * diag(G) for nE energies (Sec. 2; Eq. 2 in both passes, Eq. 8 at leaves).
 *   E       nE complex energies (eta included in the imaginary part)
 *   sigmaL  nE*nx*nx complex, row-major per energy: Sigma_L on column y=0,
 *           or NULL for the semi-infinite clean-lead closed form
 *           Phi diag(sigma_m) Phi^T (sine modes; sigma_m the root of
 *           sigma^2 - (E - eps_m) sigma + tau_m^2 = 0 with |sigma_m| < |tau_m|)
 *   sigmaR  same for Sigma_R on column y = ny-1 (NULL: closed form)
 *   diagG   out, nE*nx*ny complex, energy-major
 *   stream  cudaStream_t (NULL = legacy default stream)
 */
int find_solve_diag(find_handle* h, const double* E, int nE,
                    const double* sigmaL, const double* sigmaR,
                    double* diagG, void* stream);

/*
 * diag(G), diag(G<) and bond currents (Sec. 3.1 Eqs. 5 and 7; Sec. 3.2).
 *   Sigma< = i (fL Gamma_L + fR Gamma_R) + diag(d), Gamma = i (Sigma - Sigma^H)
 *   sigma_lesser_diag  NULL, or node-diagonal d: nx*ny complex shared by all
 *                      energies (diag_per_energy = 0) or nE*nx*ny complex
 *                      (diag_per_energy = 1)
 *   diagG, diagGl      out, nE*nx*ny complex each
 *   bond_current       out or NULL: nE*n_bonds doubles, bond i->j current
 *                      J = H_ij G<_ji - G<_ij H_ji, evaluated as
 *                      -2 H_ij Re G<_ij (exact when Sigma< is anti-Hermitian,
 *                      i.e. real fL, fR and imaginary d).  Bond order per
 *                      energy: y-bonds (x,y)->(x,y+1) [y*nx+x, y<ny-1];
 *                      x-bonds (x,y)->(x+1,y) [y*(nx-1)+x]; stencil 9 adds
 *                      (x,y)->(x+1,y+1) and (x+1,y)->(x,y+1)
 *                      [y*(nx-1)+x, y<ny-1] in that order.
 *
 * Sigma< sparsity (Sec. 4.3): without a node-diagonal term, Sigma< is zero
 * away from the contact columns y = 0 and y = ny - 1, so the upward merges of
 * clusters with no contact node skip their Sigma update (R = 0 exactly) and
 * the leaves with no contact node run their G< products over the nonzero
 * block only.  The first call that passes sigma_lesser_diag rebuilds the
 * handle's workspace and tables to run every update; they then
 * serve all later calls of the handle.
 */
int find_solve_lesser(find_handle* h, const double* E, int nE,
                      const double* sigmaL, const double* sigmaR,
                      double fL, double fR,
                      const double* sigma_lesser_diag, int diag_per_energy,
                      double* diagG, double* diagGl, double* bond_current,
                      void* stream);

/*
 * diag(G) exactly as find_solve_diag computes it, without allocating any
 * device memory.  The paper has no counterpart; this entry point exists for
 * deployment.
 *
 * Who needs it: a caller that may not or cannot call cudaMalloc -- a host
 * program whose own memory pool has already reserved the device memory, a
 * plug-in whose host application owns every device allocation, or a service
 * loop that must not allocate once it runs.  Every device buffer the solve
 * needs (resident U blocks, per-level scratch, gather and descriptor tables,
 * the status word) lives in one fixed 64 MiB array compiled into the
 * library; each GPU that loads the library holds that array until the
 * process exits.  Inputs and outputs are still the caller's (host or device
 * pointers, as for find_solve_diag).
 *
 * Limit: a mesh whose working set for one energy exceeds 64 MiB is rejected
 * with FIND_EINVAL and a message giving the size it needs (a 40x40 mesh
 * fits several energies per pass; 128x512 does not fit).  Energies are solved
 * in passes of as many as fit.
 *
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address once; make that first call before any stream
 * capture.  Every call waits for its stream to finish its work before it
 * returns (it reads back the status word), as find_solve_diag does.
 *
 * Sharing: all calls, from every handle, use the same array and leave their
 * data in it; each call uploads its own tables and clears its status word
 * before use.  Calls that overlap on the GPU (other streams or threads at the
 * same time) race on the array and return wrong results: serialise them.
 */
int find_solve_diag_static(find_handle* h, const double* E, int nE,
                           const double* sigmaL, const double* sigmaR,
                           double* diagG, void* stream);

/*
 * diag(G) and diag(G<) by the recursive Green's function method (RGF), the
 * O(Nx^3 Ny) method the paper compares FIND with (Sec. 1, Sec. 5): forward
 * and backward sweeps over the Ny transport slices of Nx nodes, FP64, the
 * energies of a pass in lockstep.  A baseline for the FIND/RGF crossover on
 * this GPU, not a second solver: closed-form leads only, Sigma< = i (fL
 * Gamma_L + fR Gamma_R) (no node-diagonal Sigma<, no bond currents).  Inputs
 * and outputs as for find_solve_lesser (host or device); the handle keeps an
 * RGF workspace of (2 Ny + 9) Nx^2 complex entries per energy of a pass
 * beside the FIND one.  FIND_ESINGULAR if a slice block is exactly singular.
 */
int find_rgf_solve_lesser(find_handle* h, const double* E, int nE, double fL, double fR,
                          double* diagG, double* diagGl, void* stream);

/* Per-kernel timing of the handle's solves (CUDA events recorded on the
 * solve's stream around every launch while profiling is on).  Kernel
 * classes: "lead", "assemble", "invert", "lu", "trsm", "zgemm32",
 * "zgemm64", "extract", "cgemm32", "cgemm64", "ffgemm32", "ffgemm64",
 * "fftrsm", "fflu", "ffinvert", "tcsplit", "tcgemm", "ldl", "ffldl" (ldl:
 * the LDL^T factorisation, flops 8 s^3 / 6; z: FP64, c: complex64,
 * ff: float-float arithmetic; 32/64: tile size; tc: the tensor-core products,
 * split into digit planes, then multiplied).  flops are the algorithmic real
 * flops of the launches (GEMM: 8 m n k per op and energy, only the tiles on
 * or above the diagonal of a complex symmetric output computed on one
 * triangle; LU: 8 s^3 / 3;
 * triangular solves: 8 s^2 b; leaf inversion: 8 n^3), bytes the algorithmic
 * DRAM bytes of the gather/extract kernels (blocks written plus source blocks
 * read) and of the plane split (operands read, planes written). */
typedef struct {
  char name[16];
  int launches;
  double ms;
  double flops;
  double bytes;
} find_kernel_stat;

/* enable = 1 clears the counters and starts recording; 0 stops. */
int find_profile(find_handle* h, int enable);

/* Waits for the recorded events and writes up to max entries; *count gets
 * the number of kernel classes. */
int find_profile_read(find_handle* h, find_kernel_stat* out, int max, int* count);

/* Peak probe of one arithmetic unit of `device` (not part of the method; the
 * roofline denominators of the FP64 and float-float kernels): kind 0 = FP32
 * FFMA, 1 = FP64 DFMA on the CUDA cores, 2 = FP64 DMMA (mma.sync m8n8k4).
 * Runs independent FMA chains on 4 CTAs of 256 threads per SM for about
 * `seconds` and writes the achieved TFLOP/s (2 flops per FMA) to *tflops.
 * Synchronises the device; returns FIND_EINVAL for a bad kind or time. */
int find_peak_probe(int kind, double seconds, int device, double* tflops);

/* Free the plan and the device workspace.  NULL is accepted. */
int find_destroy(find_handle* h);

/* Message of the handle's last failing call ("" if none); NULL handle gives
 * the message of the last failing find_create on this thread. */
const char* find_last_error(const find_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* FIND_GB300_H */
