// Complex Schur-update products on the tensor cores (tcgen05 + TMA).
//
//   D = beta C + a1 A1 op(B1) + a2 A2 op(B2)      a1, a2 = +-1, op(B) = B or B^H
//
// is the product shape of every Schur update of the passes: U = M(B,B) - L
// M(S,B) (Eq. 2), T = L Sigma(S,S) - Sigma(B,S) and R = Sigma(B,B) - L
// Sigma(S,B) + T L^H (Eq. 7, regrouped), and the leaf products G_K Sigma_K
// G_K^H.  The operands are complex128, and the FP64 path needs results as
// accurate as an FP64 product; GB300's FP64 units are slow (about 1.2
// TFLOP/s), its bf16 tensor cores fast.  The product is therefore computed by
// an error-free slice decomposition in the manner of Ozaki, Ogita, Oishi and
// Rump ("Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication", Numer. Algorithms 59, 2012):
//
//   * each row i of A = [a1 A1, a2 A2] (K concatenated) gets a power of two
//     2^ea_i above its largest |re|, |im|; each column j of op(B) = [op(B1);
//     op(B2)] gets 2^eb_j likewise;
//   * x = A_ij / 2^ea_i in (-1, 1) is written as signed base-64 digits,
//     x = 2^-5 sum_s d_s 2^-6s with d_s in [-32, 32] (the first digit has 6
//     bits, every later one 6), rounded at the last digit kept; the digit
//     planes are stored as bf16 values d_s 2^-6s (exact in bf16);
//   * the product of plane s of A and plane t of B carries the weight
//     2^-6(s+t): the pairs with s + t = q form the q-th "diagonal".  A
//     diagonal's products are integers times 2^-6q of at most 2^10 each, so
//     its sum over K <= 1024 (x 2 terms per complex part, x at most 8 pairs)
//     stays below 2^24 units and the FP32 tensor-core accumulation is EXACT;
//   * every exact diagonal is accumulated on its own, in tensor memory, and
//     added to an FP64 accumulator; the last diagonals, whose weight is below
//     the FP64 rounding of the first ones, share one FP32 accumulator;
//   * pairs with s + t >= nslices are dropped: the truncation error is about
//     (nslices + 1) 2^-6 nslices relative to 2^ea_i 2^eb_j K.
//
// Complex products use four real products per slice pair, through the
// negate-A bit of the instruction for Re = Ar Br - Ai Bi:
//   Cr += Ar Br,  Cr += (-Ai) Bi,  Ci += Ar Bi,  Ci += Ai Br.
//
// Kernels (one launch each per level stage):
//   k_tc_scale       exponent per row of A and column of op(B) (atomicMax)
//   k_tc_split_rows  digit planes of the rows of A and of B^H operands
//   k_tc_split_cols  digit planes of the columns of B operands (transposed in
//                    shared memory so that every plane row is K-contiguous)
//   k_tc_mma         one CTA per 128 x 128 complex output tile: a TMA warp
//                    streams 128 x 64 bf16 tiles (128-byte swizzle) of the
//                    planes into a 3-stage ring, one thread issues
//                    tcgen05.mma (M 128, N 128, K 16) into two double-buffered
//                    [Re | Im] FP32 accumulators in tensor memory, and four
//                    epilogue warps drain each diagonal (tcgen05.ld) into the
//                    FP64 output, applying the scales and beta C at the end.
//
// Every wait on an mbarrier is bounded by the SM clock; a wait that runs out
// records FIND_ETIMEOUT's code in the status word, and the CTA drains its
// copies and products in flight (again with a bound), frees its tensor memory
// and returns.
#include "kernels.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>

namespace findgb {

namespace {

constexpr int kTcM = 128;        // output tile rows (complex)
constexpr int kTcN = 128;        // output tile columns (complex)
constexpr int kTcK = 64;         // bf16 elements per TMA box row (128 bytes)
constexpr int kTcStages = 3;
constexpr int kTcTileBytes = kTcM * kTcK * 2;      // 16 KiB per plane tile
constexpr int kTcStageBytes = 4 * kTcTileBytes;    // Ar, Ai, Br, Bi
constexpr int kTcThreads = 192;                    // TMA warp, MMA warp, 4 epilogue warps
constexpr long long kTcSpinLimit = 4000000000ll;   // SM clocks (about 2 s)
constexpr int kNoExp = INT_MIN;                    // exponent of an all-zero row or column

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the phase with the given parity to complete; false when the
// bound runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kTcSpinLimit) return false;
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused by this layout (encoded as 1), descriptor
// version 1, swizzle mode 2 (128 bytes).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: bf16 A and B, FP32 accumulator, both
// operands K-major, M = 128, N = 128; bit 13 negates A.
__device__ __forceinline__ uint32_t idesc_bf16(bool neg_a) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format: f32
  d |= 1u << 7;                    // A format: bf16
  d |= 1u << 10;                   // B format: bf16
  d |= (neg_a ? 1u : 0u) << 13;    // negate A
  d |= (uint32_t)(kTcN >> 3) << 17;
  d |= (uint32_t)(kTcM >> 4) << 24;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Binary exponent e with |v| < 2^e for v != 0 (from the bits; v finite).
__device__ __forceinline__ int exp_above(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0ull) return INT_MIN;
  const int be = (int)(b >> 52);
  if (be == 0) {  // subnormal: 2^-1074 * mantissa
    return -1074 + 64 - __clzll((long long)b);
  }
  return be - 1023 + 1;
}

// X = round(v * 2^(P - e)) as a signed integer (|X| <= 2^P), P = 5 + 6 (nsl - 1),
// computed from the bits without the FP64 pipe; ties away from zero.  I is a
// 64-bit integer for P <= 59 (nsl <= 10), a 128-bit one above.
template <class I>
__device__ __forceinline__ I fixed_digits(double v, int e, int P) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFull;
  if (mag == 0ull) return 0;
  const int be = (int)(mag >> 52);
  unsigned long long m = mag & 0xFFFFFFFFFFFFFull;
  int ve;  // v = m * 2^ve
  if (be == 0) {
    ve = -1074;
  } else {
    m |= 1ull << 52;
    ve = be - 1075;
  }
  // X = m * 2^(ve + P - e); |v| < 2^e bounds the left shift by P - 53
  const int sh = ve + P - e;
  I x;
  if (sh >= 0) {
    x = (I)m << sh;
  } else if (sh <= -64) {
    x = 0;
  } else {
    const int r = -sh;
    x = (I)((m + (1ull << (r - 1))) >> r);
  }
  return (b >> 63) ? -x : x;
}

// The signed base-64 digits of X, least significant first, with constant
// shifts only: every digit below the top one is the balanced residue of the
// remainder mod 64, in [-32, 31], and the top digit takes what remains
// (|X| <= 2^P = 32 * 64^(nsl-1) keeps it within [-32, 32]).  Every digit is
// an integer of at most 6 bits, as the exactness of the planes' products
// requires.
template <class I>
__device__ __forceinline__ int low_digit(I& rem, bool top) {
  if (top) return (int)rem;
  const int d = (int)(((unsigned)rem + 32u) & 63u) - 32;
  rem = (rem - (I)d) >> 6;
  return d;
}

// bf16 bits of d * 2^-6s for a small integer d (|d| <= 32), exact.
__device__ __forceinline__ unsigned short digit_bf16(int d, float scale) {
  const float f = (__int_as_float(0x4B400000 + d) - 12582912.0f) * scale;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

__device__ __forceinline__ float pow2f(int k) {  // 2^k for -126 <= k <= 127
  return __uint_as_float((uint32_t)(k + 127) << 23);
}

// T 2^e2 as a double, rounded to nearest even, from the integer's bits (no
// FP64 instruction); the rare results outside the normal range go through the
// FP64 conversion.
__device__ __forceinline__ double ll_scaled(long long T, int e2) {
  if (T == 0) return 0.0;
  const unsigned long long sgn = T < 0 ? 1ull << 63 : 0ull;
  unsigned long long u = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
  int p = 63 - __clzll((long long)u);  // leading bit
  unsigned long long m;
  if (p > 52) {
    const int sh = p - 52;
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++p;
    }
  } else {
    m = u << (52 - p);
  }
  const int be = p + e2 + 1023;
  if (be < 1 || be > 2046) return ldexp((double)T, e2);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

}  // namespace

// ---------------------------------------------------------------- scales
__global__ void k_tc_scale_init(TcSlab slab, int n, int e_off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) slab.scale[(int64_t)(blockIdx.y + e_off) * slab.scale_estride + i] = kNoExp;
}

// Work items, one per CTA of 8 warps: (op, kind | part << 4, i0, k0).
// kind 0: rows i0 .. i0+7 of A1 / A2, a warp per row; kind 2: rows of a B^H
// operand (opb == 1) likewise; kind 1: columns i0 .. i0+31 of a plain B
// operand (opb == 0) over its rows k0 .. k0+63, a lane per column and 8 rows
// per warp.  Each warp reduces its maximum exponents and raises the op's with
// atomicMax.
__global__ void __launch_bounds__(256) k_tc_scale(const TcOp* __restrict__ ops,
                                                  const int4* __restrict__ items, TcSlab slab,
                                                  int e_off) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.y + e_off;
  const int4 w = items[blockIdx.x];
  const TcOp& op = ops[w.x];
  const int kind = w.y & 15, part = w.y >> 4;
  int* sc = slab.scale + (int64_t)e * slab.scale_estride;
  const int k = part ? op.k2 : op.k1;
  int best = kNoExp;
  if (kind == 1) {
    const cplx* B = part ? op.B2 + (int64_t)e * op.sb2 : op.B1 + (int64_t)e * op.sb1;
    const int ld = part ? op.ldb2 : op.ldb1;
    const int j = w.z + lane;
    const int r0 = w.w + 8 * warp, r1 = min(k, r0 + 8);
    if (j < op.n)
      for (int r = r0; r < r1; ++r) {
        const cplx v = B[(int64_t)r * ld + j];
        best = max(best, max(exp_above(v.x), exp_above(v.y)));
      }
    if (j < op.n && best != kNoExp) atomicMax(sc + op.bscale + j, best);
    return;
  }
  const int r = w.z + warp;
  const int nrows = kind == 0 ? op.m : op.n;
  if (r >= nrows) return;
  const cplx* X;
  int ld;
  if (kind == 0) {
    X = part ? op.A2 + (int64_t)e * op.sa2 : op.A1 + (int64_t)e * op.sa1;
    ld = part ? op.lda2 : op.lda1;
  } else {
    X = part ? op.B2 + (int64_t)e * op.sb2 : op.B1 + (int64_t)e * op.sb1;
    ld = part ? op.ldb2 : op.ldb1;
  }
  const cplx* row = X + (int64_t)r * ld;
  for (int j = lane; j < k; j += 32) {
    const cplx v = row[j];
    best = max(best, max(exp_above(v.x), exp_above(v.y)));
  }
  for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, off));
  if (lane == 0 && best != kNoExp) atomicMax(sc + (kind == 0 ? op.ascale : op.bscale) + r, best);
}

// The digit planes of two adjacent entries (each written only if its flag is
// set; both: one 4-byte store per plane).
template <class I>
__device__ __forceinline__ void write_digit_pair(cplx v0, cplx v1, bool m0, bool m1, int ex, int P,
                                                 int nsl, unsigned short* dst, int64_t plane_stride) {
  I r0 = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v0.x, ex, P);
  I i0 = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v0.y, ex, P);
  I r1 = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v1.x, ex, P);
  I i1 = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v1.y, ex, P);
  for (int s = nsl - 1; s >= 0; --s) {  // planes from the least significant
    const float scl = pow2f(-6 * s);
    const unsigned short a0 = digit_bf16(low_digit(r0, s == 0), scl);
    const unsigned short b0 = digit_bf16(low_digit(i0, s == 0), scl);
    const unsigned short a1 = digit_bf16(low_digit(r1, s == 0), scl);
    const unsigned short b1 = digit_bf16(low_digit(i1, s == 0), scl);
    unsigned short* pr = dst + (int64_t)(2 * s) * plane_stride;
    unsigned short* pi = dst + (int64_t)(2 * s + 1) * plane_stride;
    if (m0 && m1) {
      *reinterpret_cast<uint32_t*>(pr) = (uint32_t)a0 | ((uint32_t)a1 << 16);
      *reinterpret_cast<uint32_t*>(pi) = (uint32_t)b0 | ((uint32_t)b1 << 16);
    } else if (m0) {
      pr[0] = a0;
      pi[0] = b0;
    } else {
      pr[1] = a1;
      pi[1] = b1;
    }
  }
}

// ---------------------------------------------------------------- row planes
// Work items, one per CTA: (op, side, r0): rows r0 .. r0+7, a warp per row.
// side 0: row i of A (all K, zero padding included); side 1: row j of the
// planes of op(B), i.e. column j of op(B): this kernel writes the segments
// that come from B^H and B^T operands (contiguous rows of the stored B) and every
// zero; the segments from plain B operands are written by k_tc_split_cols.
// Each lane takes K positions.
__global__ void __launch_bounds__(256) k_tc_split_rows(const TcOp* __restrict__ ops,
                                                       const int4* __restrict__ items, TcSlab slab,
                                                       int e_off) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.y + e_off;
  const int4 w = items[blockIdx.x];
  const TcOp& op = ops[w.x];
  const int side = w.y, r = w.z + warp;
  const int rows_pad = side ? op.tiles_n * kTcN : op.mt * kTcM;
  if (r >= rows_pad) return;
  const int nsl = op.nsl, P = 5 + 6 * (nsl - 1);
  const int* sc = slab.scale + (int64_t)e * slab.scale_estride;
  const int valid = side ? op.n : op.m;
  unsigned short* base =
      (side ? slab.b : slab.a) + (int64_t)e * slab.plane_estride +
      ((int64_t)(side ? op.brow : op.arow) + r) * slab.pitch;
  const int64_t plane_stride = (int64_t)rows_pad * slab.pitch;  // between consecutive planes
  const int ex = (r < valid) ? sc[(side ? op.bscale : op.ascale) + r] : kNoExp;
  // entry k of the row, and whether this kernel writes it (segments of plain B
  // operands are k_tc_split_cols')
  auto fetch = [&](int k, cplx& v) -> bool {
    v = make_double2(0.0, 0.0);
    const bool in1 = k < op.k1, in2 = k >= op.k1p && k < op.k1p + op.k2;
    if (r >= valid || ex == kNoExp || !(in1 || in2)) return true;
    const int part = in1 ? 0 : 1;
    const int kk = in1 ? k : k - op.k1p;
    if (side == 0) {
      const cplx* A = part ? op.A2 + (int64_t)e * op.sa2 : op.A1 + (int64_t)e * op.sa1;
      const int ld = part ? op.lda2 : op.lda1;
      v = A[(int64_t)r * ld + kk];
      if (part ? op.neg2 : op.neg1) v = make_double2(-v.x, -v.y);
      return true;
    }
    const int opb = part ? op.opb2 : op.opb1;
    if (opb == 0) return false;
    const cplx* B = part ? op.B2 + (int64_t)e * op.sb2 : op.B1 + (int64_t)e * op.sb1;
    const int ld = part ? op.ldb2 : op.ldb1;
    v = B[(int64_t)r * ld + kk];
    if (opb == 1) v.y = -v.y;  // op(B) = B^H; opb 2: B^T
    return true;
  };
  // two adjacent positions per lane (kp and every segment start are multiples
  // of 64, so a pair never straddles a segment and its 4 bytes are aligned)
  for (int k = 2 * lane; k < op.kp; k += 64) {
    cplx v0, v1;
    const bool m0 = fetch(k, v0), m1 = fetch(k + 1, v1);
    if (!m0 && !m1) continue;
    if (nsl <= 10)
      write_digit_pair<long long>(v0, v1, m0, m1, ex, P, nsl, base + k, plane_stride);
    else
      write_digit_pair<__int128>(v0, v1, m0, m1, ex, P, nsl, base + k, plane_stride);
  }
}

// ---------------------------------------------------------------- column planes
template <class I>
__device__ __forceinline__ void split_cols_body(const TcOp* __restrict__ ops, const int4& w, TcSlab slab,
                                                int e, unsigned short (*tile)[32][kTcK + 2]) {
  const TcOp& op = ops[w.x];
  const int part = w.y, j0 = w.z, k0 = w.w;
  const int nsl = op.nsl, P = 5 + 6 * (nsl - 1);
  const int* sc = slab.scale + (int64_t)e * slab.scale_estride;
  const cplx* B = part ? op.B2 + (int64_t)e * op.sb2 : op.B1 + (int64_t)e * op.sb1;
  const int K = part ? op.k2 : op.k1, ld = part ? op.ldb2 : op.ldb1;
  const int kbase = part ? op.k1p : 0;  // K offset of this part in the concatenation
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = j0 + lane;
  const int ex = (j < op.n) ? sc[op.bscale + j] : kNoExp;
  // each thread: column j, K rows k0 + warp + 8 q, q = 0..7
  I xr[8], xi[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = k0 + warp + 8 * q;
    cplx v = make_double2(0.0, 0.0);
    if (j < op.n && k < K && ex != kNoExp) v = B[(int64_t)k * ld + j];
    xr[q] = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v.x, ex, P);
    xi[q] = (ex == kNoExp) ? (I)0 : fixed_digits<I>(v.y, ex, P);
  }
  const int rows_pad = op.tiles_n * kTcN;
  const int64_t plane_stride = (int64_t)rows_pad * slab.pitch;
  unsigned short* base = slab.b + (int64_t)e * slab.plane_estride + (int64_t)op.brow * slab.pitch;
  const int kw = min(kTcK, K - k0);  // positions of this block inside the part
  for (int s = nsl - 1; s >= 0; --s) {  // planes from the least significant
    const float scl = pow2f(-6 * s);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = warp + 8 * q;
      tile[0][lane][kk] = digit_bf16(low_digit(xr[q], s == 0), scl);
      tile[1][lane][kk] = digit_bf16(low_digit(xi[q], s == 0), scl);
    }
    __syncthreads();
    // 2 planes x 32 rows, a warp per row, two positions per lane (K-contiguous);
    // kbase + k0 is even, so the pairs are 4-byte aligned
    for (int pr = warp; pr < 64; pr += 8) {
      const int p = pr >> 5, jj = pr & 31;
      if (j0 + jj >= op.n) continue;  // padded rows: zero, written by k_tc_split_rows
      unsigned short* dst = base + (int64_t)(2 * s + p) * plane_stride + (int64_t)(j0 + jj) * slab.pitch + kbase + k0;
      const int kk = 2 * lane;
      if (kk + 1 < kw) {
        const uint32_t two = (uint32_t)tile[p][jj][kk] | ((uint32_t)tile[p][jj][kk + 1] << 16);
        *reinterpret_cast<uint32_t*>(dst + kk) = two;
      } else if (kk < kw) {
        dst[kk] = tile[p][jj][kk];
      }
    }
    __syncthreads();
  }
}

// Work items: (op, part, column block j0, K block k0): the 32 x 64 block
// op(B)[k0 .. k0+63][j0 .. j0+31] of a plain (opb == 0) operand B, read with
// the columns along the lanes and written K-contiguous through shared memory.
__global__ void __launch_bounds__(256) k_tc_split_cols(const TcOp* __restrict__ ops,
                                                       const int4* __restrict__ items, TcSlab slab,
                                                       int e_off) {
  __shared__ __align__(4) unsigned short tile[2][32][kTcK + 2];  // row stride 33 words
  const int e = blockIdx.y + e_off;
  const int4 w = items[blockIdx.x];
  if (ops[w.x].nsl <= 10)
    split_cols_body<long long>(ops, w, slab, e, tile);
  else
    split_cols_body<__int128>(ops, w, slab, e, tile);
}

// ---------------------------------------------------------------- the product
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_mma(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
             const TcOp* __restrict__ ops, const int* __restrict__ tile_op, TcSlab slab,
             int* __restrict__ status, int e_off) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  // 1024-byte aligned ring of stages (the 128-byte swizzle atom)
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[kTcStages], empty_bar[kTcStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x, e = blockIdx.y + e_off;
  const TcOp& op = ops[tile_op[t]];
  const int local = t - op.tile0;
  const int tm = local / op.tiles_n, tn = local % op.tiles_n;
  const int nsl = op.nsl, nexact = op.nexact;
  const int ngroups = nexact + (nsl > nexact ? 1 : 0);
  const int ksteps = op.kp / kTcK;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&empty_bar[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 4);  // one arrival per epilogue warp
    }
    mbar_init(&drain_bar, 1);
    abort_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base_sh))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  // the pair (s, t) sequence: group g < nexact is the diagonal s + t = g;
  // the last group holds every diagonal nexact .. nsl - 1
  auto group_pairs = [&](int g, int idx, int& s, int& tt) -> bool {
    const int q0 = g < nexact ? g : nexact, q1 = g < nexact ? g : nsl - 1;
    int c = 0;
    for (int q = q0; q <= q1; ++q)
      for (int a = 0; a <= q; ++a) {
        if (a >= nsl || q - a >= nsl) continue;
        if (c == idx) { s = a; tt = q - a; return true; }
        ++c;
      }
    return false;
  };
  auto group_size = [&](int g) {
    const int q0 = g < nexact ? g : nexact, q1 = g < nexact ? g : nsl - 1;
    int c = 0;
    for (int q = q0; q <= q1; ++q) c += q + 1;
    return c;
  };

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
      const int Mpad = op.mt * kTcM, Npad = op.tiles_n * kTcN;
      int stage = 0;
      uint32_t phase = 0;
      int issued = 0;
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int np = group_size(g);
        for (int ks = 0; ks < ksteps && ok; ++ks)
          for (int p = 0; p < np && ok; ++p) {
            int s = 0, tt = 0;
            group_pairs(g, p, s, tt);
            if (issued >= kTcStages && !mbar_wait(&empty_bar[stage], phase ^ 1)) { ok = false; break; }
            if (*(volatile int*)&abort_sh) { ok = false; break; }
            unsigned char* st = smem + stage * kTcStageBytes;
            mbar_expect_tx(&full_bar[stage], kTcStageBytes);
            // odd groups run over K backwards: a group starts on the tiles the
            // previous one loaded last, while they are still in L2 (the
            // order of an exact diagonal's sum does not change its value)
            const int k = ((g & 1) ? ksteps - 1 - ks : ks) * kTcK;
            const int ra = op.arow + (2 * s) * Mpad + tm * kTcM;
            const int rb = op.brow + (2 * tt) * Npad + tn * kTcN;
            tma_load_3d(st, &mapA, &full_bar[stage], k, ra, e);
            tma_load_3d(st + kTcTileBytes, &mapA, &full_bar[stage], k, ra + Mpad, e);
            tma_load_3d(st + 2 * kTcTileBytes, &mapB, &full_bar[stage], k, rb, e);
            tma_load_3d(st + 3 * kTcTileBytes, &mapB, &full_bar[stage], k, rb + Npad, e);
            ++issued;
            if (++stage == kTcStages) { stage = 0; phase ^= 1; }
          }
      }
      if (!ok) {
        atomicMin(status + 1, 1);
        abort_sh = 1;
      }
      // copies in flight complete on their own; wait for them before leaving
      // (bounded), so that nothing lands in shared memory after exit
      for (int i = 0; i < kTcStages && i < issued; ++i) {
        // the most recent fill of each slot
        const int last = issued - 1 - i;
        const int sl = last % kTcStages;
        const uint32_t ph = (uint32_t)((last / kTcStages) & 1);
        mbar_wait(&full_bar[sl], ph);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t id_pos = idesc_bf16(false), id_neg = idesc_bf16(true);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int g = 0; g < ngroups && ok; ++g) {
        const int buf = g & 1;
        if (g >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)(((g - 2) >> 1) & 1))) { ok = false; break; }
        tc_fence_after();
        const uint32_t dr = tmem + buf * 256, di = dr + 128;
        const int np = group_size(g);
        bool first = true;
        for (int ks = 0; ks < ksteps && ok; ++ks)
          for (int p = 0; p < np && ok; ++p) {
            if (!mbar_wait(&full_bar[stage], phase)) { ok = false; break; }
            if (*(volatile int*)&abort_sh) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + stage * kTcStageBytes);
            const uint64_t ar = sdesc_sw128(sa), ai = sdesc_sw128(sa + kTcTileBytes);
            const uint64_t br = sdesc_sw128(sa + 2 * kTcTileBytes), bi = sdesc_sw128(sa + 3 * kTcTileBytes);
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
              const uint64_t adv = (uint64_t)((kk * 32) >> 4);  // 16 bf16 = 32 bytes
              const uint32_t acc = first && kk == 0 ? 0u : 1u;
              umma_bf16(dr, ar + adv, br + adv, id_pos, acc);
              umma_bf16(dr, ai + adv, bi + adv, id_neg, 1u);
              umma_bf16(di, ar + adv, bi + adv, id_pos, acc);
              umma_bf16(di, ai + adv, br + adv, id_pos, 1u);
            }
            first = false;
            umma_commit(&empty_bar[stage]);  // the slot is free once these products finish
            if (++stage == kTcStages) { stage = 0; phase ^= 1; }
          }
        if (ok) umma_commit(&acc_full[buf]);
      }
      if (!ok) {
        atomicMin(status + 1, 2);
        abort_sh = 1;
      }
      // every product issued has finished before tensor memory is released
      umma_commit(&drain_bar);
      mbar_wait(&drain_bar, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue: warps 2..5; a warp reads tensor-memory lanes 32 (warp % 4) ..
    // The diagonals are summed as an exact fixed-point integer, kept in the
    // output's own 16 bytes per entry (two int64) between groups: group g's
    // value is k 2^-6g with k an integer (the last, inexact group: rounded at
    // 2^-6g), and T = sum_g k_g 2^(6 (G - g)), G the last group, |T| < 2^61.
    // The last group converts T 2^(ea + eb - 10 - 6 G) to FP64 and adds
    // beta C: one FP64 operation per entry in all.
    const int quad = warp & 3;
    const int row = quad * 32 + lane;
    const int gi = tm * kTcM + row;
    const bool row_ok = gi < op.m;
    const int* sc = slab.scale + (int64_t)e * slab.scale_estride;
    const int ea = row_ok ? sc[op.ascale + gi] : kNoExp;
    cplx* Drow = op.D + (int64_t)e * op.sd + (int64_t)(row_ok ? gi : 0) * op.ldd;
    longlong2* Trow = reinterpret_cast<longlong2*>(Drow);
    const cplx* Crow = op.C ? op.C + (int64_t)e * op.sc + (int64_t)(row_ok ? gi : 0) * op.ldc : nullptr;
    const int G = ngroups - 1;
    bool ok = true;
    for (int g = 0; g < ngroups; ++g) {
      const int buf = g & 1;
      const bool last = g == G;
      const float up = pow2f(6 * g);       // v 2^6g is the integer k (exactly, g < nexact)
      const int shift = 6 * (G - g);
      if (!mbar_wait(&acc_full[buf], (uint32_t)((g >> 1) & 1))) { ok = false; break; }
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + buf * 256;
      for (int c0 = 0; c0 < kTcN; c0 += 16) {
        const int gj0 = tn * kTcN + c0;
        longlong2 t[16];
        if (row_ok && g > 0) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            if (gj0 + jj < op.n) t[jj] = Trow[gj0 + jj];
        }
        float vr[16], vi[16];
        __syncwarp();
        tmem_ld16(trow + c0, vr);
        tmem_ld16(trow + 128 + c0, vi);
        tmem_wait_ld();
        if (row_ok) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) {
            const int gj = gj0 + jj;
            if (gj >= op.n) continue;
            const long long kr = (long long)__float2int_rn(vr[jj] * up);
            const long long ki = (long long)__float2int_rn(vi[jj] * up);
            long long Tr = (long long)((unsigned long long)kr << shift);
            long long Ti = (long long)((unsigned long long)ki << shift);
            if (g > 0) {
              Tr += t[jj].x;
              Ti += t[jj].y;
            }
            if (!last) {
              Trow[gj] = make_longlong2(Tr, Ti);
            } else {
              const int eb = sc[op.bscale + gj];
              cplx v = make_double2(0.0, 0.0);
              if (ea != kNoExp && eb != kNoExp) {
                const int e2 = ea + eb - 10 - 6 * G;
                v = make_double2(ll_scaled(Tr, e2), ll_scaled(Ti, e2));
              }
              if (Crow) {
                const cplx c = Crow[gj];
                v.x = fma(op.beta, c.x, v.x);
                v.y = fma(op.beta, c.y, v.y);
              }
              Drow[gj] = v;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
    }
    if (!ok && lane == 0) {
      atomicMin(status + 1, 3);
      abort_sh = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool load_encode() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

}  // namespace

int tc_encode_map(void* map_out, const void* base, int64_t pitch_elems, int64_t rows,
                  int64_t energies, int64_t estride_bytes) {
  if (!load_encode()) return 1;
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(map_out);
  std::memset(m, 0, sizeof(CUtensorMap));
  cuuint64_t dims[3] = {(cuuint64_t)pitch_elems, (cuuint64_t)rows, (cuuint64_t)energies};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch_elems * 2), (cuuint64_t)estride_bytes};
  cuuint32_t box[3] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 2;
}

int tc_smem_bytes() { return kTcStages * kTcStageBytes + 1024; }

static int round_up(int x, int m) { return (x + m - 1) / m * m; }

void tc_add_op(TcBuild& b, TcOp op) {
  op.k1p = round_up(op.k1, kTcK);
  op.kp = op.k1p + round_up(op.k2, kTcK);
  op.mt = (op.m + kTcM - 1) / kTcM;
  op.tiles_n = (op.n + kTcN - 1) / kTcN;
  op.tile0 = (int)b.tile_op.size();
  op.arow = (int)b.rowsA;
  op.brow = (int)b.rowsB;
  b.rowsA += 2LL * op.nsl * op.mt * kTcM;
  b.rowsB += 2LL * op.nsl * op.tiles_n * kTcN;
  op.ascale = b.scale_ints;
  b.scale_ints += op.mt * kTcM;
  op.bscale = b.scale_ints;
  b.scale_ints += op.tiles_n * kTcN;
  b.pitch = std::max<int64_t>(b.pitch, op.kp);
  const int id = (int)b.ops.size();
  for (int t = 0; t < op.mt * op.tiles_n; ++t) b.tile_op.push_back(id);
  for (int part = 0; part < 2; ++part) {
    const cplx* A = part ? op.A2 : op.A1;
    const cplx* B = part ? op.B2 : op.B1;
    const int k = part ? op.k2 : op.k1;
    if (!A || !B || k == 0) continue;
    for (int i = 0; i < op.m; i += 8) b.scale_items.push_back(make_int4(id, 0 | (part << 4), i, 0));
    if ((part ? op.opb2 : op.opb1) == 0) {
      for (int j0 = 0; j0 < op.n; j0 += 32)
        for (int k0 = 0; k0 < k; k0 += kTcK) {
          b.scale_items.push_back(make_int4(id, 1 | (part << 4), j0, k0));
          b.col_items.push_back(make_int4(id, part, j0, k0));
        }
    } else {
      for (int j = 0; j < op.n; j += 8) b.scale_items.push_back(make_int4(id, 2 | (part << 4), j, 0));
    }
  }
  for (int i = 0; i < op.mt * kTcM; i += 8) b.row_items.push_back(make_int4(id, 0, i, 0));
  for (int j = 0; j < op.tiles_n * kTcN; j += 8) b.row_items.push_back(make_int4(id, 1, j, 0));
  b.ops.push_back(op);
}

static int64_t align1k(int64_t x) { return (x + 1023) & ~int64_t(1023); }

int64_t tc_slab_bytes(const TcBuild& b, int64_t* offA, int64_t* offB, int64_t* offS) {
  int64_t o = 0;
  if (offA) *offA = o;
  o = align1k(o + b.rowsA * b.pitch * 2);
  if (offB) *offB = o;
  o = align1k(o + b.rowsB * b.pitch * 2);
  if (offS) *offS = o;
  o = align1k(o + (int64_t)b.scale_ints * 4);
  return o;
}

int64_t tc_op_slab_bytes(int m, int n, int k1, int k2, int nsl) {
  const int64_t kp = round_up(k1, kTcK) + round_up(k2, kTcK);
  const int64_t rows = 2LL * nsl * (round_up(m, kTcM) + round_up(n, kTcN));
  return rows * kp * 2 + 4LL * (round_up(m, kTcM) + round_up(n, kTcN));
}
int tc_tile_m() { return kTcM; }
int tc_tile_n() { return kTcN; }
int tc_tile_k() { return kTcK; }

void launch_tc_split(const TcLaunch& L, const TcOp* ops, const int4* scale_items, int nscale,
                     const int4* row_items, int nrow, const int4* col_items, int ncol, int nE,
                     cudaStream_t st, int e_off) {
  if (nE == 0) return;
  // exponents start below every value (atomicMax raises them)
  k_tc_scale_init<<<dim3((L.scale_ints + 255) / 256, nE), 256, 0, st>>>(L.slab, L.scale_ints, e_off);
  if (nscale) k_tc_scale<<<dim3(nscale, nE), 256, 0, st>>>(ops, scale_items, L.slab, e_off);
  if (nrow) k_tc_split_rows<<<dim3(nrow, nE), 256, 0, st>>>(ops, row_items, L.slab, e_off);
  if (ncol) k_tc_split_cols<<<dim3(ncol, nE), 256, 0, st>>>(ops, col_items, L.slab, e_off);
}

void launch_tc_mma(const TcLaunch& L, const TcOp* ops, const int* tile_op, int ntiles, int* status,
                   int nE, cudaStream_t st, int e_off) {
  if (ntiles == 0 || nE == 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tc_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes());
    attr_set = true;
  }
  k_tc_mma<<<dim3(ntiles, nE), kTcThreads, tc_smem_bytes(), st>>>(
      *reinterpret_cast<const CUtensorMap*>(L.mapA), *reinterpret_cast<const CUtensorMap*>(L.mapB), ops,
      tile_op, L.slab, status, e_off);
}

void launch_tc_gemm(const TcLaunch& L, const TcOp* ops, const int4* scale_items, int nscale,
                    const int4* row_items, int nrow, const int4* col_items, int ncol,
                    const int* tile_op, int ntiles, int* status, int nE, cudaStream_t st,
                    int e_off) {
  launch_tc_split(L, ops, scale_items, nscale, row_items, nrow, col_items, ncol, nE, st, e_off);
  launch_tc_mma(L, ops, tile_op, ntiles, status, nE, st, e_off);
}

}  // namespace findgb
