// CUDA kernels of the FIND passes (complex; FP64, float-float or complex64
// arithmetic on complex128 operands).
//
//   k_lead_modes / k_lead_dense  lead self-energy closed form (per energy)
//   k_assemble    gather M = [U_1 A_12; A_21 U_2] (and Sigma_M) ordered [S, B]
//                 (Procedures updateBoundaryNodes / updateAdjacentNodes)
//   k_lu          pivoted LU of M(S,S) in place, column by column (one CTA
//                 per op and energy; FP64)
//   k_lu_panel    the same in float-float, in panels of 4 columns; leaves its
//                 factors as float-float words for k_trsm
//   k_trsm        L = M(B,S) M(S,S)^{-1} (Eq. 13) by two triangular sweeps,
//                 row blocks spread over CTAs (FP64, or float-float reading
//                 complex128 or float-float factors)
//   k_invert      pivoted Gauss-Jordan inverse of the bordered leaf system
//                 (in global memory, or held in shared memory when it fits;
//                 FP64 or float-float)
//   k_zgemm       grouped complex GEMM on 32x32 or 64x64 tiles (FP64,
//                 float-float, or complex64): U = M(B,B) - L M(S,B) (Eq. 2),
//                 R = Sigma(B,B) - L Sigma(S,B) + (L Sigma(S,S) - Sigma(B,S)) L^H
//                 (Eq. 7 regrouped), and the leaf products G_K Sigma_K G_K^H
//   k_extract     diag G, diag G<, bond currents from the bordered leaves
#include "kernels.cuh"

#include <cfloat>
#include <climits>
#include <type_traits>

namespace findgb {

// ---------------------------------------------------------------- complex helpers
__device__ __forceinline__ cplx cmk(double x, double y) { return make_double2(x, y); }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return cmk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return cmk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return cmk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cplx cconj(cplx a) { return cmk(a.x, -a.y); }
__device__ __forceinline__ cplx cscale(cplx a, double s) { return cmk(a.x * s, a.y * s); }
// c + a * b with four fused multiply-adds
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
// c - a * b
__device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx c) {
  c.x = fma(-a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(-a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}
// 1 / z by Smith's scaled algorithm (R. L. Smith, CACM 5(8), 1962): divide by
// the larger of |re|, |im| first so that no intermediate overflows.
__device__ __forceinline__ cplx crecip(cplx z) {
  double a = z.x, b = z.y;
  if (fabs(a) >= fabs(b)) {
    double r = b / a, d = a + b * r;
    return cmk(1.0 / d, -r / d);
  } else {
    double r = a / b, d = a * r + b;
    return cmk(r / d, -1.0 / d);
  }
}
// principal square root from the polar half-angle identities
__device__ __forceinline__ cplx csqrt_principal(cplx z) {
  double r = hypot(z.x, z.y);
  if (r == 0.0) return cmk(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return cmk(t, z.y / (2.0 * t));
  return cmk(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// Float-float ("df32") arithmetic: a real x is carried as hi + lo, two
// floats with |lo| <= ulp(hi)/2 (about 48 significant bits), following
// Dekker (1971) and Knuth's error-free two-sum; complex values as float4
// (re.hi, re.lo, im.hi, im.lo).  On GB300 the FP32 pipes run about 70 times
// the FP64 rate, so a multiply-add carried this way (12 FP32 operations per
// real product) is several times faster than FP64 at nearly its accuracy.
// Split a double into hi + lo floats without the (slow) FP64 pipe: hi keeps
// the sign, the exponent and the top 23 fraction bits (truncated); lo is the
// remaining 29 fraction bits, x - hi exactly, converted to float (rounded to
// 24 bits) and scaled by 2^(e - 1075).  Values outside the float normal range
// (zero included) take the FP64 conversions.
__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ffull);
  if (e < 1023 - 126 || e > 1023 + 127) {
    if ((b << 1) == 0ull) {  // +-0 (padding, the zeros of sparse blocks): the
      h = __uint_as_float((unsigned int)(b >> 32));  // same words as below
      l = 0.0f;
      return;
    }
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
    return;
  }
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  h = __uint_as_float(sign | ((unsigned int)(e - 1023 + 127) << 23) | (unsigned int)(mant >> 29));
  float lf = (float)(unsigned int)(mant & 0x1FFFFFFFull);
  const int pe = e - 1075 + 127;  // biased float exponent of 2^(e - 1075)
  lf = (pe > 0) ? lf * __uint_as_float((unsigned int)pe << 23) : ldexpf(lf, e - 1075);
  l = sign ? -lf : lf;
}
__device__ __forceinline__ double df_join(float h, float l) { return (double)h + (double)l; }
// (ch, cl) += (ah, al) * (bh, bl): the product's exact high part, its rounding
// error by fma, the two cross terms; the sum by an error-free two-sum whose
// error joins the low word.  Normalised once at the end of a reduction.
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& ch, float& cl) {
  const float ph = ah * bh;
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float s = ch + ph;
  const float bb = s - ch;
  const float e = (ch - (s - bb)) + (ph - bb);
  cl = cl + (e + pl);
  ch = s;
}
__device__ __forceinline__ void df_norm(float& h, float& l) {
  const float t = h + l;
  l = l - (t - h);
  h = t;
}
__device__ __forceinline__ float fneg_if(float x, bool neg) {
  return __int_as_float(__float_as_int(x) ^ (neg ? (int)0x80000000 : 0));
}
// v (negated when neg) in float-float; df_split is odd in its argument, so
// negating the words afterwards is exact and needs no FP64 instruction
__device__ __forceinline__ float4 df_load(cplx v, bool neg) {
  float4 r;
  df_split(v.x, r.x, r.y);
  df_split(v.y, r.z, r.w);
  r.x = fneg_if(r.x, neg);
  r.y = fneg_if(r.y, neg);
  r.z = fneg_if(r.z, neg);
  r.w = fneg_if(r.w, neg);
  return r;
}
// c + a * b, complex float-float
__device__ __forceinline__ float4 df_cfma(float4 a, float4 b, float4 c) {
  df_mac(a.x, a.y, b.x, b.y, c.x, c.y);
  df_mac(-a.z, -a.w, b.z, b.w, c.x, c.y);
  df_mac(a.x, a.y, b.z, b.w, c.z, c.w);
  df_mac(a.z, a.w, b.x, b.y, c.z, c.w);
  return c;
}
__device__ __forceinline__ cplx df_wide(float4 v) {
  df_norm(v.x, v.y);
  df_norm(v.z, v.w);
  return make_double2(df_join(v.x, v.y), df_join(v.z, v.w));
}

// ---------------------------------------------------------------- lead self-energy
// sigma_m(E): root of sigma^2 - (E - eps_m) sigma + tau_m^2 = 0 with |sigma| < |tau|.
__global__ void k_lead_modes(const cplx* __restrict__ E, int nE, const double* __restrict__ eps,
                             const double* __restrict__ tau, int nx, cplx* __restrict__ out) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nE * nx) return;
  int e = idx / nx, m = idx % nx;
  cplx w = cmk(E[e].x - eps[m], E[e].y);
  double t2 = tau[m] * tau[m];
  cplx disc = cmk(w.x * w.x - w.y * w.y - 4.0 * t2, 2.0 * w.x * w.y);
  cplx d = csqrt_principal(disc);
  cplx r1 = cscale(cadd(w, d), 0.5), r2 = cscale(csub(w, d), 0.5);
  double a1 = r1.x * r1.x + r1.y * r1.y, a2 = r2.x * r2.x + r2.y * r2.y;
  out[idx] = (a1 < a2) ? r1 : r2;
}

// Sigma[e][x1][x2] = sum_m phi[x1][m] sigma[e][m] phi[x2][m]
__global__ void k_lead_dense(const cplx* __restrict__ sig, const double* __restrict__ phi, int nx,
                             cplx* __restrict__ out) {
  int e = blockIdx.y;
  int x1 = blockIdx.x;
  const cplx* s = sig + (int64_t)e * nx;
  for (int x2 = threadIdx.x; x2 < nx; x2 += blockDim.x) {
    cplx acc = cmk(0, 0);
    for (int m = 0; m < nx; ++m) {
      double w = phi[x1 * nx + m] * phi[x2 * nx + m];
      acc.x = fma(w, s[m].x, acc.x);
      acc.y = fma(w, s[m].y, acc.y);
    }
    out[((int64_t)e * nx + x1) * nx + x2] = acc;
  }
}

// ---------------------------------------------------------------- original entries
// A_ij = E delta_ij - H_ij - Sigma_L,ij - Sigma_R,ij  (Sec. 1)
__device__ __forceinline__ cplx a_orig(const DevProblem& P, int e, int i, int j) {
  const int nx = P.nx;
  int xi = i % nx, yi = i / nx, xj = j % nx, yj = j / nx;
  cplx v = cmk(0, 0);
  if (i == j) {
    v = cmk(P.E[e].x - (P.onsite0 + P.V[i]), P.E[e].y);
  } else {
    int dx = abs(xi - xj), dy = abs(yi - yj);
    if (dx + dy == 1) v.x = P.t;
    else if (P.stencil == 9 && dx == 1 && dy == 1) v.x = P.tp;
  }
  if (yi == 0 && yj == 0) v = csub(v, P.sigL[((int64_t)e * nx + xi) * nx + xj]);
  if (yi == P.ny - 1 && yj == P.ny - 1) v = csub(v, P.sigR[((int64_t)e * nx + xi) * nx + xj]);
  return v;
}

// Sigma<_ij = i (fL Gamma_L + fR Gamma_R)_ij + d_i delta_ij, Gamma = i (Sigma - Sigma^H)
__device__ __forceinline__ cplx s_orig(const DevProblem& P, int e, int i, int j) {
  const int nx = P.nx;
  int xi = i % nx, yi = i / nx, xj = j % nx, yj = j / nx;
  cplx v = cmk(0, 0);
  if (yi == 0 && yj == 0) {
    cplx a = P.sigL[((int64_t)e * nx + xi) * nx + xj];
    cplx b = P.sigL[((int64_t)e * nx + xj) * nx + xi];
    v = cadd(v, cscale(csub(a, cconj(b)), -P.fL));
  }
  if (yi == P.ny - 1 && yj == P.ny - 1) {
    cplx a = P.sigR[((int64_t)e * nx + xi) * nx + xj];
    cplx b = P.sigR[((int64_t)e * nx + xj) * nx + xi];
    v = cadd(v, cscale(csub(a, cconj(b)), -P.fR));
  }
  if (i == j && P.dles) v = cadd(v, P.dles[(int64_t)e * P.dles_estride + i]);
  return v;
}

// ---------------------------------------------------------------- assembly
// A warp per (row of an op, group of kAsmEnergies energies), kAsmRows rows per
// CTA: the row's position entries (which source block and index, or the
// original A and Sigma<) do not depend on the energy, so they are read once
// and reused for every energy of the group.  Rows are 20-1000 entries long; a
// warp per row keeps short rows from leaving most of a CTA idle.
constexpr int kAsmEnergies = 4;
constexpr int kAsmRows = 8;

__global__ void __launch_bounds__(256, 3) k_assemble(const AsmOp* __restrict__ ops,
                                                  const int* __restrict__ row_op,
                                                  const Pos* __restrict__ pos, DevProblem P,
                                                  int lesser, int e_off, int nE, int nrows) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * kAsmRows + (threadIdx.x >> 5);  // a warp per row
  if (r >= nrows) return;
  const AsmOp& op = ops[row_op[r]];
  const int n = op.n;
  const int p = r - op.row0;
  const Pos pp = pos[op.pos + p];
  const int e_lo = blockIdx.y * kAsmEnergies, e_hi = min(nE, e_lo + kAsmEnergies);
  const int d = pp.src == 1 ? op.d1 : (pp.src == 2 ? op.d2 : 0);
  // Sigma_M of an op whose nodes carry no Sigma< is zero and not read: skipped
  const bool les = lesser && op.sig;
  for (int q = lane; q < n; q += 32) {
    const Pos pq = pos[op.pos + q];
    if (pp.src != 0 && pq.src == pp.src) {
      // the group's source entries first (independent loads in flight), then
      // the stores
      const cplx* U = pp.src == 1 ? op.u1 : op.u2;
      const cplx* R = pp.src == 1 ? op.r1 : op.r2;
      const int64_t off0 = (int64_t)pp.idx * d + pq.idx, dd = (int64_t)d * d;
      cplx vu[kAsmEnergies], vr[kAsmEnergies];
#pragma unroll
      for (int u = 0; u < kAsmEnergies; ++u) {
        const int e = e_lo + u + e_off;
        if (e_lo + u < e_hi) {
          vu[u] = U[e * dd + off0];
          if (les) vr[u] = R ? R[e * dd + off0] : cmk(0, 0);
        }
      }
#pragma unroll
      for (int u = 0; u < kAsmEnergies; ++u) {
        const int e = e_lo + u + e_off;
        if (e_lo + u < e_hi) {
          cplx* Mrow = op.M + (int64_t)e * op.estride + (int64_t)p * n;
          Mrow[q] = vu[u];
          if (les) Mrow[(int64_t)n * n + q] = vr[u];
        }
      }
    } else {
      for (int ee = e_lo; ee < e_hi; ++ee) {
        const int e = ee + e_off;
        cplx* Mrow = op.M + (int64_t)e * op.estride + (int64_t)p * n;
        Mrow[q] = a_orig(P, e, pp.node, pq.node);
        if (les) Mrow[(int64_t)n * n + q] = s_orig(P, e, pp.node, pq.node);
      }
    }
  }
}

// ---------------------------------------------------------------- arithmetic of the
// in-place factorisations.  FP64: entries stay complex128.  Float-float: the
// kernel rewrites its block in place as (re.hi, re.lo, im.hi, im.lo) floats
// (the same 16 bytes per entry), works on that, and writes complex128 back at
// the end.  Pivot magnitudes use |re| + |im| (high words for float-float);
// pivot reciprocals are taken in FP64 (Smith) and split.
template <bool DF>
struct GA;

template <>
struct GA<false> {
  typedef cplx T;
  typedef double M;  // pivot magnitude
  __device__ __forceinline__ static T from(cplx v) { return v; }
  __device__ __forceinline__ static cplx to(T v) { return v; }
  __device__ __forceinline__ static double mag(T v) { return fabs(v.x) + fabs(v.y); }
  __device__ __forceinline__ static T zero() { return cmk(0, 0); }
  __device__ __forceinline__ static T scale(T a, T b) { return cmul(a, b); }
  __device__ __forceinline__ static T fms(T f, T r, T v) { return cfms(f, r, v); }
  __device__ __forceinline__ static bool is_zero(T v) { return v.x == 0.0 && v.y == 0.0; }
};

template <>
struct GA<true> {
  typedef float4 T;
  typedef float M;   // pivot magnitude: compared in float, no FP64 instruction
  __device__ __forceinline__ static T from(cplx v) { return df_load(v, false); }
  __device__ __forceinline__ static cplx to(T v) { return df_wide(v); }
  __device__ __forceinline__ static float mag(T v) { return fabsf(v.x) + fabsf(v.z); }
  __device__ __forceinline__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ static T scale(T a, T b) {
    T r = df_cfma(a, b, make_float4(0.f, 0.f, 0.f, 0.f));
    df_norm(r.x, r.y);
    df_norm(r.z, r.w);
    return r;
  }
  __device__ __forceinline__ static T fms(T f, T r, T v) {
    T o = df_cfma(make_float4(-f.x, -f.y, -f.z, -f.w), r, v);
    df_norm(o.x, o.y);
    df_norm(o.z, o.w);
    return o;
  }
  __device__ __forceinline__ static bool is_zero(T v) { return v.x == 0.f && v.z == 0.f; }
};

// Block-wide argmax of mag over rows k..s-1 of column k (largest magnitude,
// first index on ties); returns the row.
template <class X, class T>
__device__ __forceinline__ int pivot_row(const T* a, int ld, int k, int s, typename X::M* red_v, int* red_i,
                                         int* sh_p) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  typedef typename X::M M;
  M best = M(-1);
  int bi = INT_MAX;
  for (int i = k + tid; i < s; i += blockDim.x) {
    M mg = X::mag(a[(int64_t)i * ld + k]);
    if (mg > best) { best = mg; bi = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    M ob = __shfl_down_sync(0xffffffffu, best, off);
    int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
  __syncthreads();
  if (warp == 0) {
    best = lane < nwarp ? red_v[lane] : M(-1);
    bi = lane < nwarp ? red_i[lane] : INT_MAX;
    for (int off = 16; off > 0; off >>= 1) {
      M ob = __shfl_down_sync(0xffffffffu, best, off);
      int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) *sh_p = (bi == INT_MAX) ? k : bi;
  }
  __syncthreads();
  return *sh_p;
}

// row[j] = fms(f, rk[j], row[j]) for j = j0 + lane, j0 + lane + 32, ... < s
// (row[skip] reads as zero).  Float-float keeps four loads in flight per lane
// before the arithmetic (measured faster); FP64 loads one at a time (more
// registers cost it occupancy).  Each entry sees exactly one fms either way.
template <class X, class T>
__device__ __forceinline__ void row_update(T* row, const T* rk, T f, int j0, int s, int lane,
                                           int skip) {
  constexpr int U = std::is_same<typename X::M, float>::value ? 4 : 1;
  for (int jb = j0 + lane; jb < s; jb += 32 * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jb + 32 * u;
      if (j < s) v[u] = (j == skip) ? X::zero() : row[j];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = jb + 32 * u;
      if (j < s) row[j] = X::fms(f, rk[j], v[u]);
    }
  }
}

// ---------------------------------------------------------------- inversion
// Gauss-Jordan with partial pivoting, in place on the leading s x s block of
// a (leading dimension ld); colk, rowk: s entries of scratch, piv: s ints.
// An exactly zero pivot records the energy in *status and continues with a
// zero reciprocal.
constexpr int kInvThreads = 512;

template <class X, class T>
__device__ void gauss_jordan(T* a, int ld, int s, T* colk, T* rowk, int* piv, int* status,
                             int energy) {
  __shared__ typename X::M red_v[32];
  __shared__ int red_i[32];
  __shared__ int sh_p;
  __shared__ T sh_pinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int k = 0; k < s; ++k) {
    const int p = pivot_row<X>(a, ld, k, s, red_v, red_i, &sh_p);
    if (tid == 0) piv[k] = p;
    if (p != k)
      for (int j = tid; j < s; j += blockDim.x) {
        T t0 = a[(int64_t)k * ld + j];
        a[(int64_t)k * ld + j] = a[(int64_t)p * ld + j];
        a[(int64_t)p * ld + j] = t0;
      }
    __syncthreads();
    if (tid == 0) {  // the pivot reciprocal, once per step, in FP64 (Smith)
      const T pv = a[(int64_t)k * ld + k];
      cplx pinv = cmk(0, 0);
      if (X::is_zero(pv)) atomicMin(status, energy);
      else pinv = crecip(X::to(pv));
      sh_pinv = X::from(pinv);
    }
    __syncthreads();
    const T pinv = sh_pinv;
    for (int j = tid; j < s; j += blockDim.x) {
      T v = (j == k) ? pinv : X::scale(a[(int64_t)k * ld + j], pinv);
      rowk[j] = v;
      a[(int64_t)k * ld + j] = v;
    }
    for (int i = tid; i < s; i += blockDim.x) colk[i] = (i == k) ? X::zero() : a[(int64_t)i * ld + k];
    __syncthreads();
    for (int i = warp; i < s; i += nwarp) {
      if (i == k) continue;
      row_update<X>(a + (int64_t)i * ld, rowk, colk[i], 0, s, lane, k);
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = s - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < s; i += blockDim.x) {
        T t0 = a[(int64_t)i * ld + k];
        a[(int64_t)i * ld + k] = a[(int64_t)i * ld + p];
        a[(int64_t)i * ld + p] = t0;
      }
    __syncthreads();
  }
}

// Gauss-Jordan as above, blocked by panels of PW pivot steps: inside a panel
// each step updates only the panel's own columns and its pivot row; the
// other columns take the panel's PW steps together once it is done (the
// multipliers of every row kept in coef, the scaled pivot rows in prow).
// Every entry sees the same operations in the same order as in
// gauss_jordan, so the result is identical; the block crosses memory once per
// panel instead of once per step.  Shared memory: prow PW x s, coef s x PW.
template <class X, int PW, class T>
__device__ void gauss_jordan_panel(T* a, int ld, int s, T* prow, T* coef, int* piv, int* status,
                                   int energy) {
  __shared__ typename X::M red_v[32];
  __shared__ int red_i[32];
  __shared__ int sh_p;
  __shared__ T sh_pinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int nt = blockDim.x;
  for (int k0 = 0; k0 < s; k0 += PW) {
    const int w = min(PW, s - k0), k1 = k0 + w;
    for (int t = 0; t < w; ++t) {
      const int k = k0 + t;
      const int p = pivot_row<X>(a, ld, k, s, red_v, red_i, &sh_p);
      if (tid == 0) piv[k] = p;
      if (p != k) {  // whole rows, with the multipliers of their pending steps
        for (int j = tid; j < s; j += nt) {
          T t0 = a[(int64_t)k * ld + j];
          a[(int64_t)k * ld + j] = a[(int64_t)p * ld + j];
          a[(int64_t)p * ld + j] = t0;
        }
        for (int q = tid; q < t; q += nt) {
          T t0 = coef[k * PW + q];
          coef[k * PW + q] = coef[p * PW + q];
          coef[p * PW + q] = t0;
        }
      }
      __syncthreads();
      // the pivot row takes the panel's earlier steps on its other columns
      for (int j = tid; j < s; j += nt) {
        if (j >= k0 && j < k1) continue;
        T v = a[(int64_t)k * ld + j];
        for (int q = 0; q < t; ++q) v = X::fms(coef[k * PW + q], prow[q * s + j], v);
        a[(int64_t)k * ld + j] = v;
      }
      __syncthreads();
      if (tid == 0) {  // the pivot reciprocal, once per step, in FP64 (Smith)
        const T pv = a[(int64_t)k * ld + k];
        cplx pinv = cmk(0, 0);
        if (X::is_zero(pv)) atomicMin(status, energy);
        else pinv = crecip(X::to(pv));
        sh_pinv = X::from(pinv);
      }
      __syncthreads();
      const T pinv = sh_pinv;
      for (int j = tid; j < s; j += nt) {
        T v = (j == k) ? pinv : X::scale(a[(int64_t)k * ld + j], pinv);
        prow[t * s + j] = v;
        a[(int64_t)k * ld + j] = v;
      }
      __syncthreads();
      // every other row: its multiplier, and this step on the panel's columns
      for (int i = tid; i < s; i += nt) {
        if (i == k) continue;
        T* row = a + (int64_t)i * ld;
        const T m = row[k];
        coef[i * PW + t] = m;
        for (int j = k0; j < k1; ++j) row[j] = X::fms(m, prow[t * s + j], j == k ? X::zero() : row[j]);
      }
      __syncthreads();
    }
    // the panel's steps on every other column, a warp per row (a pivot row
    // of the panel takes only the steps after its own)
    for (int i = warp; i < s; i += nwarp) {
      const int q0 = (i >= k0 && i < k1) ? i - k0 + 1 : 0;
      if (q0 >= w) continue;
      T c[PW];
#pragma unroll
      for (int q = 0; q < PW; ++q)
        if (q >= q0 && q < w) c[q] = coef[i * PW + q];
      T* row = a + (int64_t)i * ld;
      for (int j = lane; j < s; j += 64) {  // two independent chains in flight
        const int j2 = j + 32;
        const bool on0 = !(j >= k0 && j < k1), on1 = j2 < s && !(j2 >= k0 && j2 < k1);
        T v0 = on0 ? row[j] : X::zero(), v1 = on1 ? row[j2] : X::zero();
#pragma unroll
        for (int q = 0; q < PW; ++q)
          if (q >= q0 && q < w) {
            if (on0) v0 = X::fms(c[q], prow[q * s + j], v0);
            if (on1) v1 = X::fms(c[q], prow[q * s + j2], v1);
          }
        if (on0) row[j] = v0;
        if (on1) row[j2] = v1;
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int k = s - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k)
      for (int i = tid; i < s; i += nt) {
        T t0 = a[(int64_t)i * ld + k];
        a[(int64_t)i * ld + k] = a[(int64_t)i * ld + p];
        a[(int64_t)i * ld + p] = t0;
      }
    __syncthreads();
  }
}

// Rewrites the leading s x s block of a complex128 matrix in the storage of
// arithmetic X (a no-op for FP64), or back.
template <class X>
__device__ __forceinline__ void to_work(cplx* a, int ld, int s) {
  if (!std::is_same<typename X::T, cplx>::value) {
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
      const int i = idx / s, j = idx % s;
      cplx v = a[(int64_t)i * ld + j];
      reinterpret_cast<typename X::T*>(a)[(int64_t)i * ld + j] = X::from(v);
    }
    __syncthreads();
  }
}
template <class X>
__device__ __forceinline__ void from_work(cplx* a, int ld, int s) {
  if (!std::is_same<typename X::T, cplx>::value) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
      const int i = idx / s, j = idx % s;
      typename X::T v = reinterpret_cast<typename X::T*>(a)[(int64_t)i * ld + j];
      a[(int64_t)i * ld + j] = X::to(v);
    }
  }
}

// Inversion in global memory, one CTA per (op, energy): blocked in panels of
// kInvPanel steps up to kInvPanelMax rows (the panel's rows and multipliers
// in shared memory), step by step above.
constexpr int kInvPanel = 4;
constexpr int kInvPanelMax = 1024;

template <bool DF>
__global__ void __launch_bounds__(kInvThreads) k_invert(const InvOp* __restrict__ ops,
                                                        int* __restrict__ status, int e_base,
                                                        int e_off, int panel) {
  typedef GA<DF> X;
  typedef typename X::T T;
  const InvOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  if (s == 0) return;
  cplx* a = op.M + (int64_t)e * op.estride;
  extern __shared__ double2 inv_smem[];
  to_work<X>(a, ld, s);
  if (panel) {  // the launch's largest block fits the panel layout
    T* prow = reinterpret_cast<T*>(inv_smem);
    T* coef = prow + (int64_t)kInvPanel * s;
    int* piv = reinterpret_cast<int*>(coef + (int64_t)kInvPanel * s);
    gauss_jordan_panel<X, kInvPanel>(reinterpret_cast<T*>(a), ld, s, prow, coef, piv, status, e_base + e);
  } else {
    T* colk = reinterpret_cast<T*>(inv_smem);
    T* rowk = colk + s;
    int* piv = reinterpret_cast<int*>(rowk + s);
    gauss_jordan<X>(reinterpret_cast<T*>(a), ld, s, colk, rowk, piv, status, e_base + e);
  }
  from_work<X>(a, ld, s);
}

// Inversion with the whole block held in shared memory (s <= kInvSmemMax):
// no global traffic between the load and the store.
constexpr int kInvSmemMax = 112;

template <bool DF>
__global__ void __launch_bounds__(kInvThreads) k_invert_smem(const InvOp* __restrict__ ops,
                                                             int* __restrict__ status, int e_base,
                                                             int e_off) {
  typedef GA<DF> X;
  typedef typename X::T T;
  const InvOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  if (s == 0) return;
  cplx* g = op.M + (int64_t)e * op.estride;
  extern __shared__ double2 invs_smem[];
  T* a = reinterpret_cast<T*>(invs_smem);  // s x s, leading dimension s
  T* colk = a + (int64_t)s * s;
  T* rowk = colk + s;
  int* piv = reinterpret_cast<int*>(rowk + s);
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx % s;
    a[idx] = X::from(g[(int64_t)i * ld + j]);
  }
  __syncthreads();
  gauss_jordan<X>(a, s, s, colk, rowk, piv, status, e_base + e);
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx % s;
    g[(int64_t)i * ld + j] = X::to(a[idx]);
  }
}

// ---------------------------------------------------------------- LU factorisation
// Right-looking LU with partial pivoting (largest |re| + |im|, first index on
// ties) of the leading s x s block, in place: P M = L U with unit-lower L
// below the diagonal.  Whole rows are interchanged, LAPACK style; piv[k] is
// the row exchanged with row k at step k.  One CTA per (op, energy).  An
// exactly zero pivot records the energy in *status and continues.
template <bool DF>
__global__ void __launch_bounds__(kInvThreads) k_lu(const InvOp* __restrict__ ops,
                                                    int* __restrict__ status, int e_base,
                                                    int e_off) {
  typedef GA<DF> X;
  typedef typename X::T T;
  const InvOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  if (s == 0) return;
  cplx* g = op.M + (int64_t)e * op.estride;
  int* piv = op.piv + (int64_t)e * op.piv_estride;
  extern __shared__ double2 lu_smem[];
  T* rowk = reinterpret_cast<T*>(lu_smem);
  __shared__ typename X::M red_v[32];
  __shared__ int red_i[32];
  __shared__ int sh_p;
  __shared__ T sh_pinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  to_work<X>(g, ld, s);
  T* a = reinterpret_cast<T*>(g);
  for (int k = 0; k < s; ++k) {
    const int p = pivot_row<X>(a, ld, k, s, red_v, red_i, &sh_p);
    if (tid == 0) piv[k] = p;
    if (p != k)
      for (int j = tid; j < s; j += blockDim.x) {
        T t0 = a[(int64_t)k * ld + j];
        a[(int64_t)k * ld + j] = a[(int64_t)p * ld + j];
        a[(int64_t)p * ld + j] = t0;
      }
    __syncthreads();
    if (tid == 0) {  // the pivot reciprocal, once per step, in FP64 (Smith)
      const T pv = a[(int64_t)k * ld + k];
      cplx pinv = cmk(0, 0);
      if (X::is_zero(pv)) atomicMin(status, e_base + e);
      else pinv = crecip(X::to(pv));
      sh_pinv = X::from(pinv);
    }
    __syncthreads();
    const T pinv = sh_pinv;
    for (int j = k + 1 + tid; j < s; j += blockDim.x) rowk[j] = a[(int64_t)k * ld + j];
    for (int i = k + 1 + tid; i < s; i += blockDim.x)
      a[(int64_t)i * ld + k] = X::scale(a[(int64_t)i * ld + k], pinv);
    __syncthreads();
    for (int i = k + 1 + warp; i < s; i += nwarp) {
      T* row = a + (int64_t)i * ld;
      row_update<X>(row, rowk, row[k], k + 1, s, lane, -1);
    }
    __syncthreads();
  }
  from_work<X>(g, ld, s);
}

// Float-float LU, blocked by panels of PW columns: each panel is factorised
// column by column (pivot search, full-row interchange, scaling, update of the
// panel's own later columns); then its U rows are completed over the trailing
// columns (kept in shared memory) and the trailing block takes one rank-PW
// update.  Every entry sees the same operations in the same order as in
// k_lu, so the factors are identical; the trailing block, which at large s
// does not fit in L2, crosses HBM once per panel instead of once per column.
constexpr int kLuPanel = 4;

template <int PW>
__global__ void __launch_bounds__(kInvThreads, 2) k_lu_panel(const InvOp* __restrict__ ops,
                                                            int* __restrict__ status, int e_base,
                                                            int e_off) {
  typedef GA<true> X;
  typedef X::T T;
  const InvOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  if (s == 0) return;
  cplx* g = op.M + (int64_t)e * op.estride;
  int* piv = op.piv + (int64_t)e * op.piv_estride;
  extern __shared__ double2 lu_smem[];
  T* urow = reinterpret_cast<T*>(lu_smem);  // PW x s: the panel's U rows
  __shared__ X::M red_v[32];
  __shared__ int red_i[32];
  __shared__ int sh_p;
  __shared__ T sh_pinv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int nt = blockDim.x;
  to_work<X>(g, ld, s);
  T* a = reinterpret_cast<T*>(g);
  for (int k0 = 0; k0 < s; k0 += PW) {
    const int w = min(PW, s - k0), k1 = k0 + w;
    for (int k = k0; k < k1; ++k) {
      const int p = pivot_row<X>(a, ld, k, s, red_v, red_i, &sh_p);
      if (tid == 0) piv[k] = p;
      if (p != k)
        for (int j = tid; j < s; j += nt) {
          T t0 = a[(int64_t)k * ld + j];
          a[(int64_t)k * ld + j] = a[(int64_t)p * ld + j];
          a[(int64_t)p * ld + j] = t0;
        }
      __syncthreads();
      if (tid == 0) {  // the pivot reciprocal, once per step, in FP64 (Smith)
        const T pv = a[(int64_t)k * ld + k];
        cplx pinv = cmk(0, 0);
        if (X::is_zero(pv)) atomicMin(status, e_base + e);
        else pinv = crecip(X::to(pv));
        sh_pinv = X::from(pinv);
      }
      __syncthreads();
      const T pinv = sh_pinv;
      for (int i = k + 1 + tid; i < s; i += nt) {
        // scale the column, then update the rest of this row inside the panel
        T* row = a + (int64_t)i * ld;
        const T l = X::scale(row[k], pinv);
        row[k] = l;
        for (int c = k + 1; c < k1; ++c) row[c] = X::fms(l, a[(int64_t)k * ld + c], row[c]);
      }
      __syncthreads();
    }
    // the panel's U rows over the trailing columns, one column per thread
    for (int j = k1 + tid; j < s; j += nt) {
      for (int t = 0; t < w; ++t) {
        T u = a[(int64_t)(k0 + t) * ld + j];
        for (int t2 = 0; t2 < t; ++t2)
          u = X::fms(a[(int64_t)(k0 + t) * ld + k0 + t2], urow[t2 * s + j], u);
        urow[t * s + j] = u;
        a[(int64_t)(k0 + t) * ld + j] = u;
      }
    }
    __syncthreads();
    // the trailing block: one rank-w update, a warp per row
    for (int i = k1 + warp; i < s; i += nwarp) {
      T* row = a + (int64_t)i * ld;
      T l[PW];
#pragma unroll
      for (int t = 0; t < PW; ++t)
        if (t < w) l[t] = row[k0 + t];
      int j = k1 + lane;
      for (; j + 32 < s; j += 64) {  // two independent chains in flight
        T v0 = row[j], v1 = row[j + 32];
#pragma unroll
        for (int t = 0; t < PW; ++t)
          if (t < w) {
            v0 = X::fms(l[t], urow[t * s + j], v0);
            v1 = X::fms(l[t], urow[t * s + j + 32], v1);
          }
        row[j] = v0;
        row[j + 32] = v1;
      }
      if (j < s) {
        T v = row[j];
#pragma unroll
        for (int t = 0; t < PW; ++t)
          if (t < w) v = X::fms(l[t], urow[t * s + j], v);
        row[j] = v;
      }
    }
    __syncthreads();
  }
  // the factors stay float-float words: their only reader, the float-float
  // TRSM, takes them as they are (k_trsm<true, true>)
}

// ---------------------------------------------------------------- LDL^T factorisation
// Block-wide maximum of f(i) over i in [i0, i1) (first index on ties); every
// thread gets (value, index); index -1 for an empty range.
template <class Fn>
__device__ __forceinline__ void block_argmax(int i0, int i1, Fn f, double* red_v, int* red_i,
                                             double& best_out, int& idx_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  double best = -1.0;
  int bi = INT_MAX;
  for (int i = i0 + tid; i < i1; i += blockDim.x) {
    const double m = f(i);
    if (m > best) { best = m; bi = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  __syncthreads();  // red_v / red_i may still be read from a previous call
  if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
  __syncthreads();
  best = red_v[0];
  bi = red_i[0];
  for (int w = 1; w < nwarp; ++w)
    if (red_v[w] > best || (red_v[w] == best && red_i[w] < bi)) { best = red_v[w]; bi = red_i[w]; }
  best_out = best;
  idx_out = bi == INT_MAX ? -1 : bi;
}

__device__ __forceinline__ double cabs1(cplx v) { return fabs(v.x) + fabs(v.y); }

// Symmetric indefinite factorisation of the complex symmetric M(S,S) with
// the diagonal pivoting of Bunch and Kaufman (Math. Comp. 31, 1977): at step k
// with alpha = (1 + sqrt 17) / 8 and lambda the largest |.| below the
// diagonal in column k (row r), take a 1x1 pivot a_kk when |a_kk| >= alpha
// lambda, or when |a_kk| sigma >= alpha lambda^2 with sigma the largest
// off-diagonal |.| in row/column r; else a 1x1 pivot a_rr when |a_rr| >=
// alpha sigma; else the 2x2 pivot on {k, r}.  |.| is |re| + |im|.  Only the
// lower triangle is read and updated (half the flops of the LU, Sec. 4.2).
// FP64, or float-float (the block rewritten in place as float-float words
// during the factorisation, like k_lu).  Blocks of up to kLdlPanelMax rows
// are factorised in panels (ldl_panel, below), larger ones step by step.
// On exit: P M P^T = T D T^T with T unit lower, stored below the diagonal
// (zero at the sub-diagonal of each 2x2 block) and mirrored above it (the
// forward sweep of k_trsm reads T^T there), ones on the diagonal; D in dv
// (diagonal, then the 2x2 sub-diagonals); piv[j] the row and column
// interchanged with j at its step (LU convention), kind[j] = 0 for a 1x1
// block, 1 / 2 for the first / second index of a 2x2 block.  A pivot block
// that is exactly singular records the energy in *status.
template <class T>
__device__ __forceinline__ T neg_of(T v);
template <>
__device__ __forceinline__ cplx neg_of(cplx v) { return cmk(-v.x, -v.y); }
template <>
__device__ __forceinline__ float4 neg_of(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// The same factorisation blocked by panels of at least PW columns: inside a
// panel no step updates the trailing triangle; a column takes the panel's
// earlier steps when it is needed (the candidate pivot column k, and row and
// column r for the pivot test, formed aside in wk and wr), and the trailing
// triangle takes all of the panel's steps at once at its end.  The unscaled
// pivot columns are kept in C (s x (PW + 1), by row), so a symmetric
// interchange swaps two rows of C with the rows of A.  Each entry sees the
// same products as in the step-by-step kernel, but an entry that an
// interchange moves across the diagonal takes its update from the other
// triangle's operands (l_j c_i for l_i c_j), so the factors agree with it to
// rounding, not bit for bit; the pivot decisions use the same updated values.
template <class X, int PW, class T>
__device__ void ldl_panel(T* a, int ld, int s, int* piv, int* kind, cplx* dv, T* C, T* wk, T* wr,
                          int* status, int energy, double* red_v, int* red_i) {
  constexpr int CW = PW + 1;  // a panel ends after PW columns, or PW + 1 with a closing 2x2 block
  __shared__ int lcol[CW];
  __shared__ int sh_kp, sh_step;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const int nt = blockDim.x;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  auto A = [&](int i, int j) -> T& { return a[(int64_t)i * ld + j]; };
  // entry (i, j), i >= j, of the lower triangle with the panel's steps applied
  auto upd = [&](int i, int j, int nc) {
    T v = A(i, j);
    for (int c = 0; c < nc; ++c) v = X::fms(A(i, lcol[c]), C[j * CW + c], v);
    return v;
  };
  int k = 0;
  while (k < s) {
    int nc = 0;
    while (k < s && nc < PW) {
      for (int i = k + tid; i < s; i += nt) wk[i] = upd(i, k, nc);
      __syncthreads();
      double colmax;
      int imax;
      block_argmax(k + 1, s, [&](int i) { return (double)X::mag(wk[i]); }, red_v, red_i, colmax, imax);
      const double absakk = (double)X::mag(wk[k]);
      int kp = k, step = 1;
      if (colmax > 0.0 && absakk < alpha * colmax) {
        for (int j = k + tid; j < s; j += nt)
          wr[j] = j == k ? wk[imax] : (j < imax ? upd(imax, j, nc) : upd(j, imax, nc));
        __syncthreads();
        double rm1, rm2;
        int i1, i2;
        block_argmax(k, imax, [&](int j) { return (double)X::mag(wr[j]); }, red_v, red_i, rm1, i1);
        block_argmax(imax + 1, s, [&](int j) { return (double)X::mag(wr[j]); }, red_v, red_i, rm2, i2);
        const double rowmax = fmax(rm1, rm2);
        if (absakk * rowmax >= alpha * colmax * colmax) {
          kp = k;
        } else if ((double)X::mag(wr[imax]) >= alpha * rowmax) {
          kp = imax;
        } else {
          kp = imax;
          step = 2;
        }
      }
      if (tid == 0) { sh_kp = kp; sh_step = step; }
      __syncthreads();
      kp = sh_kp;
      step = sh_step;
      const int kk = k + step - 1;
      if (!(step == 1 && kp != k))  // column k stays: it takes its updated values
        for (int i = k + tid; i < s; i += nt) A(i, k) = wk[i];
      __syncthreads();
      if (kp != kk) {
        if (tid == 0) {
          const T t = A(kk, kk);
          A(kk, kk) = A(kp, kp);
          A(kp, kp) = t;
        }
        for (int j = kk + 1 + tid; j < kp; j += nt) {
          const T t = A(j, kk);
          A(j, kk) = A(kp, j);
          A(kp, j) = t;
        }
        for (int i = kp + 1 + tid; i < s; i += nt) {
          const T t = A(i, kk);
          A(i, kk) = A(i, kp);
          A(i, kp) = t;
        }
        for (int j = tid; j < kk; j += nt) {
          const T t = A(kk, j);
          A(kk, j) = A(kp, j);
          A(kp, j) = t;
        }
        for (int c = tid; c < nc; c += nt) {
          const T t = C[kk * CW + c];
          C[kk * CW + c] = C[kp * CW + c];
          C[kp * CW + c] = t;
        }
      }
      if (tid == 0) {
        piv[k] = (step == 1) ? kp : k;
        kind[k] = step == 1 ? 0 : 1;
        if (step == 2) {
          piv[k + 1] = kp;
          kind[k + 1] = 2;
        }
      }
      __syncthreads();
      if (step == 1) {
        if (kp != k) {  // the new column k takes the panel's steps
          for (int i = k + tid; i < s; i += nt) wk[i] = upd(i, k, nc);
          __syncthreads();
          for (int i = k + tid; i < s; i += nt) A(i, k) = wk[i];
          __syncthreads();
        }
        const cplx d = X::to(A(k, k));
        const bool zero = d.x == 0.0 && d.y == 0.0;
        const T r = X::from(zero ? cmk(0, 0) : crecip(d));
        if (tid == 0) {
          dv[k] = d;
          dv[s + k] = cmk(0, 0);
          if (zero) atomicMin(status, energy);
          lcol[nc] = k;
        }
        for (int i = k + 1 + tid; i < s; i += nt) {
          const T c = A(i, k);
          C[i * CW + nc] = c;
          A(i, k) = X::scale(c, r);
        }
      } else {
        for (int i = k + 1 + tid; i < s; i += nt) wk[i] = upd(i, k + 1, nc);
        __syncthreads();
        for (int i = k + 1 + tid; i < s; i += nt) A(i, k + 1) = wk[i];
        __syncthreads();
        const cplx d11 = X::to(A(k, k)), d21 = X::to(A(k + 1, k)), d22 = X::to(A(k + 1, k + 1));
        const cplx det = csub(cmul(d11, d22), cmul(d21, d21));
        const bool zero = det.x == 0.0 && det.y == 0.0;
        const cplx r = zero ? cmk(0, 0) : crecip(det);
        const T e11 = X::from(cmul(d22, r)), e22 = X::from(cmul(d11, r));
        const T e21 = X::from(cmk(-(cmul(d21, r).x), -(cmul(d21, r).y)));
        if (tid == 0) {
          dv[k] = d11;
          dv[k + 1] = d22;
          dv[s + k] = d21;
          dv[s + k + 1] = cmk(0, 0);
          if (zero) atomicMin(status, energy);
          lcol[nc] = k;
          lcol[nc + 1] = k + 1;
        }
        for (int i = k + 2 + tid; i < s; i += nt) {
          const T x1 = A(i, k), x2 = A(i, k + 1);
          C[i * CW + nc] = x1;
          C[i * CW + nc + 1] = x2;
          A(i, k) = X::fms(x2, neg_of(e21), X::scale(x1, e11));
          A(i, k + 1) = X::fms(x2, neg_of(e22), X::scale(x1, e21));
        }
        __syncthreads();
        if (tid == 0) A(k + 1, k) = X::zero();  // T is the identity on the 2x2 block
      }
      __syncthreads();
      nc += step;
      k += step;
    }
    // the panel's steps on the trailing triangle, a warp per row
    for (int i = k + warp; i < s; i += nwarp) {
      T l[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c)
        if (c < nc) l[c] = A(i, lcol[c]);
      T* row = a + (int64_t)i * ld;
      for (int j = k + lane; j <= i; j += 32) {
        T v = row[j];
#pragma unroll
        for (int c = 0; c < CW; ++c)
          if (c < nc) v = X::fms(l[c], C[j * CW + c], v);
        row[j] = v;
      }
    }
    __syncthreads();
  }
}
constexpr int kLdlPanel = 4;
constexpr int kLdlPanelMax = 1024;

template <bool DF>
__global__ void __launch_bounds__(kInvThreads, 2) k_ldl(const InvOp* __restrict__ ops,
                                                     int* __restrict__ status, int e_base,
                                                     int e_off, int panel) {
  typedef GA<DF> X;
  typedef typename X::T T;
  const InvOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  if (s == 0) return;
  cplx* g = op.M + (int64_t)e * op.estride;
  int* piv = op.piv + (int64_t)e * op.piv_estride;
  int* kind = piv + s;
  cplx* dv = op.dv + (int64_t)e * op.estride;
  extern __shared__ double2 ldl_smem[];
  T* c1 = reinterpret_cast<T*>(ldl_smem);  // unscaled pivot columns
  T* c2 = c1 + s;
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int sh_kp, sh_step;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const double alpha = (1.0 + sqrt(17.0)) / 8.0;
  to_work<X>(g, ld, s);
  T* a = reinterpret_cast<T*>(g);
  auto A = [&](int i, int j) -> T& { return a[(int64_t)i * ld + j]; };
  auto mag = [&](int i, int j) { return (double)X::mag(A(i, j)); };
  if (panel) {  // the launch's largest block fits C, wk and wr in shared memory
    T* C = reinterpret_cast<T*>(ldl_smem);
    T* wk = C + (int64_t)s * (kLdlPanel + 1);
    T* wr = wk + s;
    ldl_panel<X, kLdlPanel>(a, ld, s, piv, kind, dv, C, wk, wr, status, e_base + e, red_v, red_i);
  }
  int k = panel ? s : 0;
  while (k < s) {
    double colmax;
    int imax;
    block_argmax(k + 1, s, [&](int i) { return mag(i, k); }, red_v, red_i, colmax, imax);
    const double absakk = mag(k, k);
    int kp = k, step = 1;
    if (colmax > 0.0 && absakk < alpha * colmax) {
      double rm1, rm2;
      int i1, i2;
      block_argmax(k, imax, [&](int j) { return mag(imax, j); }, red_v, red_i, rm1, i1);
      block_argmax(imax + 1, s, [&](int j) { return mag(j, imax); }, red_v, red_i, rm2, i2);
      const double rowmax = fmax(rm1, rm2);
      if (absakk * rowmax >= alpha * colmax * colmax) {
        kp = k;
      } else if (mag(imax, imax) >= alpha * rowmax) {
        kp = imax;
      } else {
        kp = imax;
        step = 2;
      }
    }
    if (tid == 0) { sh_kp = kp; sh_step = step; }
    __syncthreads();
    kp = sh_kp;
    step = sh_step;
    const int kk = k + step - 1;
    if (kp != kk) {
      // symmetric interchange of kk and kp on the lower triangle, and of the
      // two rows of the columns already eliminated
      if (tid == 0) {
        const T t = A(kk, kk);
        A(kk, kk) = A(kp, kp);
        A(kp, kp) = t;
      }
      for (int j = kk + 1 + tid; j < kp; j += blockDim.x) {
        const T t = A(j, kk);
        A(j, kk) = A(kp, j);
        A(kp, j) = t;
      }
      for (int i = kp + 1 + tid; i < s; i += blockDim.x) {
        const T t = A(i, kk);
        A(i, kk) = A(i, kp);
        A(i, kp) = t;
      }
      for (int j = tid; j < kk; j += blockDim.x) {
        const T t = A(kk, j);
        A(kk, j) = A(kp, j);
        A(kp, j) = t;
      }
    }
    if (tid == 0) {
      piv[k] = (step == 1) ? kp : k;
      kind[k] = step == 1 ? 0 : 1;
      if (step == 2) {
        piv[k + 1] = kp;
        kind[k + 1] = 2;
      }
    }
    __syncthreads();
    if (step == 1) {
      // the pivot reciprocal in FP64 (Smith), split for float-float
      const cplx d = X::to(A(k, k));
      const bool zero = d.x == 0.0 && d.y == 0.0;
      const T r = X::from(zero ? cmk(0, 0) : crecip(d));
      if (tid == 0) {
        dv[k] = d;
        dv[s + k] = cmk(0, 0);
        if (zero) atomicMin(status, e_base + e);
      }
      for (int i = k + 1 + tid; i < s; i += blockDim.x) {
        const T c = A(i, k);
        c1[i] = c;
        A(i, k) = X::scale(c, r);
      }
      __syncthreads();
      // a_ij -= l_i c_j for k < j <= i, a warp per row
      for (int i = k + 1 + warp; i < s; i += nwarp) {
        const T li = A(i, k);
        T* row = a + (int64_t)i * ld;
        for (int j = k + 1 + lane; j <= i; j += 32) row[j] = X::fms(li, c1[j], row[j]);
      }
    } else {
      const cplx d11 = X::to(A(k, k)), d21 = X::to(A(k + 1, k)), d22 = X::to(A(k + 1, k + 1));
      const cplx det = csub(cmul(d11, d22), cmul(d21, d21));
      const bool zero = det.x == 0.0 && det.y == 0.0;
      const cplx r = zero ? cmk(0, 0) : crecip(det);
      const T e11 = X::from(cmul(d22, r)), e22 = X::from(cmul(d11, r));
      const T e21 = X::from(cmk(-(cmul(d21, r).x), -(cmul(d21, r).y)));
      if (tid == 0) {
        dv[k] = d11;
        dv[k + 1] = d22;
        dv[s + k] = d21;
        dv[s + k + 1] = cmk(0, 0);
        if (zero) atomicMin(status, e_base + e);
      }
      for (int i = k + 2 + tid; i < s; i += blockDim.x) {
        const T x1 = A(i, k), x2 = A(i, k + 1);
        c1[i] = x1;
        c2[i] = x2;
        // l1 = x1 e11 + x2 e21, l2 = x1 e21 + x2 e22
        A(i, k) = X::fms(x2, neg_of(e21), X::scale(x1, e11));
        A(i, k + 1) = X::fms(x2, neg_of(e22), X::scale(x1, e21));
      }
      __syncthreads();
      if (tid == 0) A(k + 1, k) = X::zero();  // T is the identity on the 2x2 block
      for (int i = k + 2 + warp; i < s; i += nwarp) {
        const T l1 = A(i, k), l2 = A(i, k + 1);
        T* row = a + (int64_t)i * ld;
        for (int j = k + 2 + lane; j <= i; j += 32) row[j] = X::fms(l2, c2[j], X::fms(l1, c1[j], row[j]));
      }
    }
    __syncthreads();
    k += step;
  }
  // unit diagonal, and T^T mirrored into the upper triangle
  const T one = X::from(cmk(1.0, 0.0));
  for (int idx = tid; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx % s;
    if (i == j) A(i, i) = one;
    else if (j > i) A(i, j) = A(j, i);
  }
  // the factors leave as complex128 (the solves split them when they read)
  from_work<X>(g, ld, s);
}

// ---------------------------------------------------------------- grouped complex GEMM
// Operands are complex128 in memory; CT is the arithmetic type: double2 (FP64
// path) or float2 (complex64 arithmetic of the mixed path, operands rounded
// when staged in shared memory, the epilogue adds beta * C in FP64).
template <class CT>
struct Cx;

template <>
struct Cx<double2> {
  __device__ __forceinline__ static double2 zero() { return make_double2(0.0, 0.0); }
  __device__ __forceinline__ static double2 load(cplx v, bool neg) {
    return neg ? make_double2(-v.x, -v.y) : v;
  }
  __device__ __forceinline__ static double2 fma(double2 a, double2 b, double2 c) { return cfma(a, b, c); }
  __device__ __forceinline__ static cplx wide(double2 v) { return v; }
  __device__ __forceinline__ static void renorm(double2&) {}
};

template <>
struct Cx<float2> {
  __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
  __device__ __forceinline__ static float2 load(cplx v, bool neg) {
    return make_float2(fneg_if((float)v.x, neg), fneg_if((float)v.y, neg));
  }
  __device__ __forceinline__ static float2 fma(float2 a, float2 b, float2 c) {
    c.x = fmaf(a.x, b.x, c.x);
    c.x = fmaf(-a.y, b.y, c.x);
    c.y = fmaf(a.x, b.y, c.y);
    c.y = fmaf(a.y, b.x, c.y);
    return c;
  }
  __device__ __forceinline__ static cplx wide(float2 v) { return make_double2(v.x, v.y); }
  __device__ __forceinline__ static void renorm(float2&) {}
};

template <>
struct Cx<float4> {
  __device__ __forceinline__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ static float4 load(cplx v, bool neg) { return df_load(v, neg); }
  __device__ __forceinline__ static float4 fma(float4 a, float4 b, float4 c) { return df_cfma(a, b, c); }
  __device__ __forceinline__ static cplx wide(float4 v) { return df_wide(v); }
  __device__ __forceinline__ static void renorm(float4& v) {
    df_norm(v.x, v.y);
    df_norm(v.z, v.w);
  }
};

// Tile BM x BN per CTA, BK deep; each thread owns a 4 x 4 block of outputs at
// rows ty + i*BM/4, cols tx + j*BN/4.  alpha is folded into the A tile.
template <int BM, int BN, int BK, class CT>
// float-float: at most 128 registers, so 16 warps share an SM (2 CTAs of the
// 64x64 tile, 8 of the 32x32 one)
__global__ void __launch_bounds__((BM / 4) * (BN / 4), sizeof(CT) == 16 ? (BM == 64 ? 2 : 8) : 1)
    k_zgemm(const GemmOp* __restrict__ ops,
                                                               const int* __restrict__ tile_op,
                                                               int e_off, int sym_mask) {
  typedef Cx<CT> X;
  constexpr int NT = (BM / 4) * (BN / 4);
  constexpr int RS = BM / 4, CS = BN / 4;
  __shared__ CT As[BK][BM + 1];
  __shared__ CT Bs[BK][BN + 1];
  const int t = blockIdx.x, e = blockIdx.y + e_off;
  const GemmOp& op = ops[tile_op[t]];
  const int local = t - op.tile0;
  const int tm = local / op.tiles_n, tn = local % op.tiles_n;
  const int m0 = tm * BM, n0 = tn * BN;
  // a complex symmetric output: only tiles on or above the diagonal work,
  // and mirror what they compute
  const bool mirror = BM == BN && op.sym == 1 && (sym_mask & 1);
  if (mirror && tm > tn) return;
  const int tx = threadIdx.x % CS, ty = threadIdx.x / CS;
  const int M = op.m, N = op.n;
  CT acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = X::zero();

  for (int pass = 0; pass < 2; ++pass) {
    const cplx* A = pass ? op.A2 : op.A;
    const cplx* B = pass ? op.B2 : op.B;
    const int K = pass ? op.k2 : op.k;
    if (A == nullptr || K == 0) continue;
    const int lda = pass ? op.lda2 : op.lda, ldb = pass ? op.ldb2 : op.ldb;
    const int opb = pass ? op.opb2 : op.opb;
    const bool neg = (pass ? op.alpha2 : op.alpha) < 0.0;  // alpha is +1 or -1
    A += (int64_t)e * (pass ? op.sa2 : op.sa);
    B += (int64_t)e * (pass ? op.sb2 : op.sb);
    for (int k0 = 0; k0 < K; k0 += BK) {
      for (int idx = threadIdx.x; idx < BM * BK; idx += NT) {
        int i = idx / BK, kk = idx % BK;
        int gi = m0 + i, gk = k0 + kk;
        cplx v = (gi < M && gk < K) ? A[(int64_t)gi * lda + gk] : cmk(0, 0);
        As[kk][i] = X::load(v, neg);
      }
      if (opb == 0) {
        for (int idx = threadIdx.x; idx < BK * BN; idx += NT) {
          int kk = idx / BN, j = idx % BN;
          int gk = k0 + kk, gj = n0 + j;
          Bs[kk][j] = X::load((gk < K && gj < N) ? B[(int64_t)gk * ldb + gj] : cmk(0, 0), false);
        }
      } else {
        // B stored n x k: op(B) = B^H (opb 1) or B^T (opb 2)
        for (int idx = threadIdx.x; idx < BK * BN; idx += NT) {
          int j = idx / BK, kk = idx % BK;
          int gk = k0 + kk, gj = n0 + j;
          cplx v = (gk < K && gj < N) ? B[(int64_t)gj * ldb + gk] : cmk(0, 0);
          Bs[kk][j] = X::load(opb == 1 ? cconj(v) : v, false);
        }
      }
      __syncthreads();
      // the float-float step is ~800 instructions: unrolling the k loop
      // as well would outgrow the instruction cache
#pragma unroll(sizeof(CT) == 16 ? 1 : BK)
      for (int kk = 0; kk < BK; ++kk) {
        CT av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + i * RS];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + j * CS];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = X::fma(av[i], bv[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) X::renorm(acc[i][j]);
      __syncthreads();
    }
  }
  const cplx* C = op.C ? op.C + (int64_t)e * op.sc : nullptr;
  cplx* D = op.D + (int64_t)e * op.sd;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gi = m0 + ty + i * RS;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gj = n0 + tx + j * CS;
      if (gj >= N) continue;
      if (mirror && gi > gj) continue;  // the (gj, gi) thread writes this pair
      cplx v = X::wide(acc[i][j]);
      if (C) {
        cplx c = C[(int64_t)gi * op.ldc + gj];
        v.x = fma(op.beta, c.x, v.x);
        v.y = fma(op.beta, c.y, v.y);
      }
      D[(int64_t)gi * op.ldd + gj] = v;
      if (mirror && gi != gj) D[(int64_t)gj * op.ldd + gi] = v;
    }
  }
}

// ---------------------------------------------------------------- L = M(B,S) M(S,S)^{-1}
// Row block of RB rows per CTA held in shared memory.  The forward sweep
// solves Y U = M(B,S) in panels of W columns: each row solves the panel's
// own columns (scale by 1/U_jj, eliminate within the panel), then every later
// column takes a rank-W update; the backward sweep solves Z L = Y with the
// unit-lower factor the same way, right to left; the row interchanges are
// then applied as column interchanges.  DF: the row block is carried in
// float-float (factors read in FP64 and split once per use, shared by the
// RB rows).
template <bool DF>
struct TrsmArith;

template <>
struct TrsmArith<false> {
  typedef cplx T;
  __device__ __forceinline__ static T zero() { return cmk(0, 0); }
  __device__ __forceinline__ static T shfl(T v, int src) {
    return cmk(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
  }
  __device__ __forceinline__ static T in(cplx v) { return v; }
  __device__ __forceinline__ static cplx out(T v) { return v; }
  __device__ __forceinline__ static T mul(T a, cplx b) { return cmul(a, b); }
  __device__ __forceinline__ static T mul2(T a, T b) { return cmul(a, b); }
  __device__ __forceinline__ static T fms(T a, T b, T c) { return cfms(a, b, c); }
};

template <>
struct TrsmArith<true> {
  typedef float4 T;
  __device__ __forceinline__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ static T shfl(T v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
  }
  __device__ __forceinline__ static T in(cplx v) { return df_load(v, false); }
  __device__ __forceinline__ static cplx out(T v) { return df_wide(v); }
  __device__ __forceinline__ static T mul(T a, cplx b) {
    return df_cfma(a, df_load(b, false), make_float4(0.f, 0.f, 0.f, 0.f));
  }
  __device__ __forceinline__ static T mul2(T a, T b) {
    T r = df_cfma(a, b, make_float4(0.f, 0.f, 0.f, 0.f));
    df_norm(r.x, r.y);
    df_norm(r.z, r.w);
    return r;
  }
  __device__ __forceinline__ static T fms(T a, T b, T c) {
    T r = df_cfma(make_float4(-a.x, -a.y, -a.z, -a.w), b, c);
    df_norm(r.x, r.y);
    df_norm(r.z, r.w);
    return r;
  }
};

constexpr int kTrsmW = 16;       // columns per panel (8 measured slower: twice the barriers,
                                 // and half the block idle in each panel solve)
constexpr int kTrsmRowsMax = 16; // rows per CTA at most (24 measured slower)
constexpr int kPanelThreads = kTrsmW * kTrsmRowsMax;  // 8 whole warps: the block
static_assert(kPanelThreads % 32 == 0 && 32 % kTrsmW == 0, "panel lanes must tile warps");

// Entries of the LU factors of M(S,S).  FF: the float-float LU left them as
// float-float words (re.hi, re.lo, im.hi, im.lo) in the 16 bytes of each
// complex128 slot, so they are read as they are; otherwise they are
// complex128 and split on reading.
template <class X, bool FF>
__device__ __forceinline__ typename X::T fac_in(const cplx* p) {
  if constexpr (FF) return *reinterpret_cast<const float4*>(p);
  else return X::in(*p);
}
template <bool FF>
__device__ __forceinline__ cplx fac_wide(const cplx* p) {
  if constexpr (FF) return df_wide(*reinterpret_cast<const float4*>(p));
  else return *p;
}

// Y(r, i) -= sum_{t < w} Y(r, j0 + t) * F(j0 + t, i) for rows r < rows and
// columns i in [c0, c1), F the factor in a (leading dimension ld).  Threads
// take (column, row group) pairs so that narrow updates still occupy the
// block; each element sees the same operations in the same order as one
// thread per column would give it.
template <class X, bool FF, class T>
__device__ __forceinline__ void rank_update(T* Y, const cplx* a, int ld, int s, int rows, int j0,
                                            int w, int c0, int c1, int tid, int nt) {
  constexpr int WC = 8;  // factor rows held in registers at a time
  const int C = c1 - c0;
  if (C <= 0) return;
  const int tpc = C >= nt ? 1 : max(1, min(rows, nt / C));  // threads per column
  const int rpt = (rows + tpc - 1) / tpc;                   // rows per thread
  for (int it = tid; it < C * tpc; it += nt) {
    const int i = c0 + it / tpc, rg = it % tpc;
    const int r1 = min(rows, (rg + 1) * rpt);
    for (int t0 = 0; t0 < w; t0 += WC) {  // the panel's rows in order, WC at a time
      const int wc = min(WC, w - t0);
      T u[WC];
#pragma unroll
      for (int t = 0; t < WC; ++t)
        if (t < wc) u[t] = fac_in<X, FF>(a + (int64_t)(j0 + t0 + t) * ld + i);
      int r = rg * rpt;
      for (; r + 1 < r1; r += 2) {  // two independent chains in flight
        T v0 = Y[r * s + i], v1 = Y[(r + 1) * s + i];
#pragma unroll
        for (int t = 0; t < WC; ++t)
          if (t < wc) {
            v0 = X::fms(Y[r * s + j0 + t0 + t], u[t], v0);
            v1 = X::fms(Y[(r + 1) * s + j0 + t0 + t], u[t], v1);
          }
        Y[r * s + i] = v0;
        Y[(r + 1) * s + i] = v1;
      }
      if (r < r1) {
        T v = Y[r * s + i];
#pragma unroll
        for (int t = 0; t < WC; ++t)
          if (t < wc) v = X::fms(Y[r * s + j0 + t0 + t], u[t], v);
        Y[r * s + i] = v;
      }
    }
  }
}

template <bool DF, bool FF, bool LDL>
__global__ void __launch_bounds__(256) k_trsm(const TrsmOp* __restrict__ ops,
                                              const int* __restrict__ tile_op, int rb, int e_off) {
  typedef TrsmArith<DF> X;
  typedef typename X::T T;
  constexpr int W = kTrsmW;  // one panel solve and one rank-W update per barrier pair
  const TrsmOp& op = ops[tile_op[blockIdx.x]];
  const int e = blockIdx.y + e_off;
  const int s = op.s, ld = op.ld;
  const int r0 = (blockIdx.x - op.tile0) * rb;
  const int rows = min(rb, op.b - r0);
  if (s == 0 || rows <= 0) return;
  const cplx* a = op.M + (int64_t)e * op.estride;
  const int* piv = op.piv + (int64_t)e * op.piv_estride;
  extern __shared__ double2 tr_smem[];
  T* Y = reinterpret_cast<T*>(tr_smem);            // rows x s
  int* perm = reinterpret_cast<int*>(Y + (int64_t)rb * s);
  __shared__ T pan[W][W];                           // the panel's block of the factor
  __shared__ T dgl[W];                              // reciprocals of the panel's diagonal
  const int tid = threadIdx.x, nt = blockDim.x;
  if (LDL) {
    // the rows are taken in the pivoted order: entry j of M(B,S) P^T is entry
    // perm[j] of M(B,S), perm the interchanges applied in order
    if (tid == 0) {
      for (int j = 0; j < s; ++j) perm[j] = j;
      for (int j = 0; j < s; ++j) {
        int p = piv[j];
        if (p < j || p >= s) p = j;
        const int t0 = perm[j];
        perm[j] = perm[p];
        perm[p] = t0;
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < rows * s; idx += nt) {
    int r = idx / s, j = idx % s;
    Y[r * s + j] = X::in(a[(int64_t)(s + r0 + r) * ld + (LDL ? perm[j] : j)]);
  }
  // forward: Y U = B, panels of W columns left to right
  for (int j0 = 0; j0 < s; j0 += W) {
    const int w = min(W, s - j0);
    for (int idx = tid; idx < w * w; idx += nt) {
      const int t = idx / w, t2 = idx % w;
      const cplx* up = a + (int64_t)(j0 + t) * ld + j0 + t2;
      if (t == t2) {
        const cplx u = fac_wide<FF>(up);
        const bool z = (u.x == 0.0 && u.y == 0.0);  // zero only if the LU flagged it
        dgl[t] = X::in(z ? cmk(0, 0) : crecip(u));
      } else {
        pan[t][t2] = fac_in<X, FF>(up);
      }
    }
    __syncthreads();
    if (tid < kPanelThreads) {  // the panel's own columns: W lanes per row, whole warps
      const int r = tid / W, c = tid % W, grp = (tid & 31) & ~(W - 1);
      const bool act = r < rows && c < w;
      T yv = act ? Y[r * s + j0 + c] : X::zero();
      for (int t = 0; t < w; ++t) {
        if (act && c == t) yv = X::mul2(yv, dgl[t]);
        const T yt = X::shfl(yv, grp | t);  // column t of this row, final from here on
        if (act && c > t) yv = X::fms(yt, pan[t][c], yv);
      }
      if (act) Y[r * s + j0 + c] = yv;
    }
    __syncthreads();
    rank_update<X, FF>(Y, a, ld, s, rows, j0, w, j0 + w, s, tid, nt);  // the later columns
    __syncthreads();
  }
  if (LDL) {
    // W^T is the forward result; then W^T D^-1, with D's 1x1 and 2x2 blocks
    const int* kind = piv + s;
    const cplx* dv = op.dv + (int64_t)e * op.l_estride;
    cplx* Wt = op.Wt + (int64_t)e * op.l_estride;
    cplx* Yd = op.Yd + (int64_t)e * op.l_estride;
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += nt) {
      const int r = idx / s, j = idx % s;
      Wt[(int64_t)(r0 + r) * s + j] = X::out(Y[r * s + j]);
    }
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += nt) {
      const int r = idx / s, j = idx % s;
      const int kd = kind[j];
      if (kd == 0) {
        const cplx d = dv[j];
        const bool z = d.x == 0.0 && d.y == 0.0;
        Y[r * s + j] = X::mul(Y[r * s + j], z ? cmk(0, 0) : crecip(d));
      } else if (kd == 1) {
        const cplx d11 = dv[j], d22 = dv[j + 1], d21 = dv[s + j];
        const cplx det = csub(cmul(d11, d22), cmul(d21, d21));
        const bool z = det.x == 0.0 && det.y == 0.0;
        const cplx rr = z ? cmk(0, 0) : crecip(det);
        const cplx e11 = cmul(d22, rr), e22 = cmul(d11, rr);
        const cplx e21 = cmk(-cmul(d21, rr).x, -cmul(d21, rr).y);
        const cplx y1 = X::out(Y[r * s + j]), y2 = X::out(Y[r * s + j + 1]);
        Y[r * s + j] = X::in(cfma(y2, e21, cmul(y1, e11)));
        Y[r * s + j + 1] = X::in(cfma(y2, e22, cmul(y1, e21)));
      }
    }
    __syncthreads();
    for (int idx = tid; idx < rows * s; idx += nt) {
      const int r = idx / s, j = idx % s;
      Yd[(int64_t)(r0 + r) * s + j] = X::out(Y[r * s + j]);
    }
    __syncthreads();
  }
  // backward: Z L = Y with L unit lower, panels of W columns right to left
  for (int je = s; je > 0; je -= W) {
    const int j0 = max(0, je - W), w = je - j0;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int t = idx / w, t2 = idx % w;
      if (t2 < t) pan[t][t2] = fac_in<X, FF>(a + (int64_t)(j0 + t) * ld + j0 + t2);
    }
    __syncthreads();
    if (tid < kPanelThreads) {
      const int r = tid / W, c = tid % W, grp = (tid & 31) & ~(W - 1);
      const bool act = r < rows && c < w;
      T yv = act ? Y[r * s + j0 + c] : X::zero();
      for (int t = w - 1; t > 0; --t) {
        const T yt = X::shfl(yv, grp | t);
        if (act && c < t) yv = X::fms(yt, pan[t][c], yv);
      }
      if (act) Y[r * s + j0 + c] = yv;
    }
    __syncthreads();
    rank_update<X, FF>(Y, a, ld, s, rows, j0, w, 0, j0, tid, nt);  // the earlier columns
    __syncthreads();
  }
  // L = Z P: column j of the result is column perm[j] of Z
  if (tid == 0) {
    for (int j = 0; j < s; ++j) perm[j] = j;
    for (int k = s - 1; k >= 0; --k) {
      int p = piv[k];
      if (p < k || p >= s) p = k;  // a valid interchange of step k lies in [k, s)
      int t0 = perm[k];
      perm[k] = perm[p];
      perm[p] = t0;
    }
  }
  __syncthreads();
  cplx* L = op.L + (int64_t)e * op.l_estride;
  for (int idx = tid; idx < rows * s; idx += nt) {
    int r = idx / s, j = idx % s;
    L[(int64_t)(r0 + r) * s + j] = X::out(Y[r * s + perm[j]]);
  }
}

// ---------------------------------------------------------------- leaf extraction
__global__ void __launch_bounds__(256) k_extract(const ExtractOp* __restrict__ ops,
                                                 const LeafBond* __restrict__ bonds, DevProblem P,
                                                 int lesser, int want_bonds, cplx* __restrict__ diagG,
                                                 cplx* __restrict__ diagGl, double* __restrict__ J,
                                                 int64_t n_nodes, int64_t n_bonds, int e_off) {
  const ExtractOp op = ops[blockIdx.x];
  const int e = blockIdx.y + e_off;
  const cplx* K = op.K + (int64_t)e * op.estride;
  const cplx* Q = op.Q + (int64_t)e * op.estride;
  for (int i = threadIdx.x; i < op.c; i += blockDim.x) {
    int node = (op.y0 + i / op.wx) * P.nx + op.x0 + i % op.wx;
    int kk = op.nb + i;
    diagG[(int64_t)e * n_nodes + node] = K[(int64_t)kk * op.n + kk];
    if (lesser) diagGl[(int64_t)e * n_nodes + node] = Q[(int64_t)i * op.n + kk];
  }
  if (lesser && want_bonds)
    for (int b = threadIdx.x; b < op.nbond; b += blockDim.x) {
      const LeafBond lb = bonds[op.bond + b];
      cplx g = Q[(int64_t)(lb.pi - op.nb) * op.n + lb.pj];
      double h = lb.kind ? -P.tp : -P.t;  // H_ij of the bond
      J[(int64_t)e * n_bonds + lb.bond] = -2.0 * h * g.x;
    }
}

// ---------------------------------------------------------------- launchers
void launch_lead_modes(const cplx* E, int nE, const double* eps, const double* tau, int nx,
                       cplx* sig_modes, cudaStream_t st) {
  int total = nE * nx;
  k_lead_modes<<<(total + 255) / 256, 256, 0, st>>>(E, nE, eps, tau, nx, sig_modes);
}

void launch_lead_dense(const cplx* sig_modes, const double* phi, int nx, int nE, cplx* out,
                       cudaStream_t st) {
  dim3 grid(nx, nE);
  k_lead_dense<<<grid, 128, 0, st>>>(sig_modes, phi, nx, out);
}

void launch_assemble(const AsmOp* ops, const int* row_op, int nrows, const Pos* pos,
                     const DevProblem& P, int lesser, int nE, cudaStream_t st, int e_off) {
  if (nrows == 0 || nE == 0) return;
  dim3 grid((nrows + kAsmRows - 1) / kAsmRows, (nE + kAsmEnergies - 1) / kAsmEnergies);
  k_assemble<<<grid, 32 * kAsmRows, 0, st>>>(ops, row_op, pos, P, lesser, e_off, nE, nrows);
}

// Threads per block of the factorisations and inversions: every entry sees
// the same operations in the same order whatever the count (warps take rows,
// the pivot search reduces over all warps), so the results do not depend on it.
int inv_threads(int max_s) {
  return max_s <= kSmallBlock ? 128 : (max_s <= 2 * kSmallBlock ? 256 : kInvThreads);
}

void launch_invert(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
                   cudaStream_t st, int e_off, int df, int in_smem) {
  if (nops == 0 || max_s == 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    const int glob = (int)std::max((size_t)kMaxInvert * (2 * sizeof(cplx) + sizeof(int)),
                                   (size_t)kInvPanelMax * (2 * kInvPanel * sizeof(cplx) + sizeof(int)));
    const int sm = (int)((size_t)kInvSmemMax * kInvSmemMax * sizeof(cplx) +
                         (size_t)kInvSmemMax * (2 * sizeof(cplx) + sizeof(int)));
    cudaFuncSetAttribute(k_invert<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, glob);
    cudaFuncSetAttribute(k_invert<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, glob);
    cudaFuncSetAttribute(k_invert_smem<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_invert_smem<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    attr_set = true;
  }
  dim3 grid(nops, nE);
  if (in_smem) {
    size_t smem = (size_t)max_s * max_s * sizeof(cplx) + (size_t)max_s * (2 * sizeof(cplx) + sizeof(int));
    if (df)
      k_invert_smem<true><<<grid, kInvThreads, smem, st>>>(ops, status, e_base, e_off);
    else
      k_invert_smem<false><<<grid, kInvThreads, smem, st>>>(ops, status, e_base, e_off);
  } else {
    // the panels' rows and multipliers (s <= kInvPanelMax), or a row and a column
    size_t smem = max_s <= kInvPanelMax ? (size_t)max_s * (2 * kInvPanel * sizeof(cplx) + sizeof(int))
                                        : (size_t)max_s * (2 * sizeof(cplx) + sizeof(int));
    // 512 threads whatever the size: 128-thread blocks for the small bordered
    // leaves measured slower than 512-thread ones
    const int nt = kInvThreads, panel = max_s <= kInvPanelMax ? 1 : 0;
    if (df)
      k_invert<true><<<grid, nt, smem, st>>>(ops, status, e_base, e_off, panel);
    else
      k_invert<false><<<grid, nt, smem, st>>>(ops, status, e_base, e_off, panel);
  }
}

void launch_lu(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
               cudaStream_t st, int e_off, int df) {
  if (nops == 0 || max_s <= 0) return;
  dim3 grid(nops, nE);
  if (df) {
    // PW rows of the largest s of the launch (s <= kMaxInvert)
    static bool attr_set = false;
    if (!attr_set) {
      cudaFuncSetAttribute(k_lu_panel<kLuPanel>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kLuPanel * kMaxInvert * (int)sizeof(float4));
      attr_set = true;
    }
    const size_t smem = (size_t)kLuPanel * max_s * sizeof(float4);
    k_lu_panel<kLuPanel><<<grid, inv_threads(max_s), smem, st>>>(ops, status, e_base, e_off);
  } else {
    k_lu<false><<<grid, inv_threads(max_s), kMaxInvert * sizeof(cplx), st>>>(ops, status, e_base, e_off);
  }
}

int invert_smem_max() { return kInvSmemMax; }

constexpr int kTrsmSmem = 196608;

int trsm_rows_per_block(int max_s) {
  if (max_s <= 0) return kTrsmRowsMax;
  int rb = (int)((kTrsmSmem - (int64_t)max_s * 4) / ((int64_t)max_s * sizeof(cplx)));
  return rb < 1 ? 1 : (rb > kTrsmRowsMax ? kTrsmRowsMax : rb);
}

void launch_trsm(const TrsmOp* ops, const int* tile_op, int ntiles, int rb, int max_s, int nE,
                 cudaStream_t st, int df, int e_off, int ff_factors, int ldl) {
  if (ntiles == 0 || max_s == 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_trsm<false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmSmem);
    cudaFuncSetAttribute(k_trsm<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmSmem);
    cudaFuncSetAttribute(k_trsm<true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmSmem);
    cudaFuncSetAttribute(k_trsm<false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmSmem);
    cudaFuncSetAttribute(k_trsm<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrsmSmem);
    attr_set = true;
  }
  size_t smem = (size_t)rb * max_s * sizeof(cplx) + (size_t)max_s * sizeof(int);
  dim3 grid(ntiles, nE);
  const int nt = 256;  // 512 threads for blocks alone on their SM measured slower
  if (ldl && df)
    k_trsm<true, false, true><<<grid, nt, smem, st>>>(ops, tile_op, rb, e_off);
  else if (ldl)
    k_trsm<false, false, true><<<grid, nt, smem, st>>>(ops, tile_op, rb, e_off);
  else if (df && ff_factors)
    k_trsm<true, true, false><<<grid, nt, smem, st>>>(ops, tile_op, rb, e_off);
  else if (df)
    k_trsm<true, false, false><<<grid, nt, smem, st>>>(ops, tile_op, rb, e_off);
  else
    k_trsm<false, false, false><<<grid, nt, smem, st>>>(ops, tile_op, rb, e_off);
}

void launch_ldl(const InvOp* ops, int nops, int max_s, int* status, int e_base, int nE,
                cudaStream_t st, int e_off, int df) {
  if (nops == 0 || max_s <= 0) return;
  static bool attr_set = false;
  if (!attr_set) {
    const int most = std::max(2 * kMaxInvert, (kLdlPanel + 3) * kLdlPanelMax) * (int)sizeof(cplx);
    cudaFuncSetAttribute(k_ldl<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(k_ldl<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    attr_set = true;
  }
  dim3 grid(nops, nE);
  const int nt = inv_threads(max_s), panel = max_s <= kLdlPanelMax ? 1 : 0;
  // panel: C (s x (kLdlPanel + 1)), wk and wr; step by step: two unscaled columns
  const size_t smem = (size_t)max_s * (panel ? kLdlPanel + 3 : 2) * sizeof(cplx);
  if (df)
    k_ldl<true><<<grid, nt, smem, st>>>(ops, status, e_base, e_off, panel);
  else
    k_ldl<false><<<grid, nt, smem, st>>>(ops, status, e_base, e_off, panel);
}

void launch_gemm(const GemmOp* ops, const int* tile_op, int ntiles, int big, int nE,
                 cudaStream_t st, int fp32, int e_off, int sym_mask) {
  if (ntiles == 0) return;
  dim3 grid(ntiles, nE);
  if (fp32 == 2) {
    if (big)
      k_zgemm<64, 64, 8, float4><<<grid, 256, 0, st>>>(ops, tile_op, e_off, sym_mask);
    else
      k_zgemm<32, 32, 8, float4><<<grid, 64, 0, st>>>(ops, tile_op, e_off, sym_mask);
  } else if (fp32) {
    if (big)
      k_zgemm<64, 64, 16, float2><<<grid, 256, 0, st>>>(ops, tile_op, e_off, sym_mask);
    else
      k_zgemm<32, 32, 16, float2><<<grid, 64, 0, st>>>(ops, tile_op, e_off, sym_mask);
  } else {
    if (big)
      k_zgemm<64, 64, 8, double2><<<grid, 256, 0, st>>>(ops, tile_op, e_off, sym_mask);
    else
      k_zgemm<32, 32, 8, double2><<<grid, 64, 0, st>>>(ops, tile_op, e_off, sym_mask);
  }
}

void launch_extract(const ExtractOp* ops, int nops, const LeafBond* bonds, const DevProblem& P,
                    int lesser, int want_bonds, cplx* diagG, cplx* diagGl, double* J,
                    int64_t n_nodes, int64_t n_bonds, int nE, cudaStream_t st, int e_off) {
  if (nops == 0) return;
  dim3 grid(nops, nE);
  k_extract<<<grid, 256, 0, st>>>(ops, bonds, P, lesser, want_bonds, diagG, diagGl, J, n_nodes,
                                  n_bonds, e_off);
}

}  // namespace findgb
