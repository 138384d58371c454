// Kernels of the recursive Green's function (RGF) baseline: the O(Nx^3 Ny)
// method FIND is compared with (Sec. 1, Sec. 5).  A is block tridiagonal in
// the transport slices y = 0 .. Ny-1 (Nx nodes each); the blocks between
// neighbouring slices are the real symmetric tridiagonal coupling C
// (A_{y,y+1} = A_{y+1,y} = C: t on the diagonal, t' beside it for the
// 9-point stencil; A = E - H with H_ij = -t, -t').  The products with C are
// sparse (three entries per row) and run here; the dense products and the
// inversions of the slice blocks use the FIND kernels (k_zgemm, k_invert).
#include "kernels.cuh"

namespace findgb {

namespace {

__device__ __forceinline__ double c_entry(const RgfSlice& s, int a, int b) {
  const int d = abs(a - b);
  return d == 0 ? s.t : (d == 1 && s.stencil == 9 ? s.tp : 0.0);
}

}  // namespace

// M = A_yy - C X C  (X = nullptr: M = A_yy).  A_yy = E - onsite0 - V(x, y) on
// the diagonal, t between transverse neighbours, minus Sigma_L (y = 0) and
// Sigma_R (y = Ny - 1).  One CTA row of M per (row, energy).
__global__ void __launch_bounds__(256) k_rgf_block(RgfSlice s, int y, const cplx* __restrict__ X,
                                                  int64_t xstride, cplx* __restrict__ M,
                                                  int64_t mstride) {
  const int a = blockIdx.x, e = blockIdx.y, nx = s.nx;
  const cplx* Xe = X ? X + (int64_t)e * xstride : nullptr;
  cplx* row = M + (int64_t)e * mstride + (int64_t)a * nx;
  for (int b = threadIdx.x; b < nx; b += blockDim.x) {
    double re = 0.0, im = 0.0;
    if (a == b) {
      re = s.E[e].x - s.onsite0 - s.V[(int64_t)y * nx + a];
      im = s.E[e].y;
    } else if (abs(a - b) == 1) {
      re = s.t;
    }
    if (y == 0) {
      const cplx v = s.sigL[((int64_t)e * nx + a) * nx + b];
      re -= v.x;
      im -= v.y;
    }
    if (y == s.ny - 1) {
      const cplx v = s.sigR[((int64_t)e * nx + a) * nx + b];
      re -= v.x;
      im -= v.y;
    }
    if (Xe) {
      for (int p = max(0, a - 1); p <= min(nx - 1, a + 1); ++p) {
        const double cap = c_entry(s, a, p);
        if (cap == 0.0) continue;
        for (int q = max(0, b - 1); q <= min(nx - 1, b + 1); ++q) {
          const double w = cap * c_entry(s, q, b);
          if (w == 0.0) continue;
          const cplx xv = Xe[(int64_t)p * nx + q];
          re -= w * xv.x;
          im -= w * xv.y;
        }
      }
    }
    row[b] = make_double2(re, im);
  }
}

// W = sign C X (left product with the tridiagonal coupling), or with
// sandwich = 1: W = C X C.
__global__ void __launch_bounds__(256) k_rgf_cprod(RgfSlice s, const cplx* __restrict__ X,
                                                  int64_t xstride, cplx* __restrict__ Wout,
                                                  int64_t wstride, double sign, int sandwich) {
  const int a = blockIdx.x, e = blockIdx.y, nx = s.nx;
  const cplx* Xe = X + (int64_t)e * xstride;
  cplx* row = Wout + (int64_t)e * wstride + (int64_t)a * nx;
  for (int b = threadIdx.x; b < nx; b += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int p = max(0, a - 1); p <= min(nx - 1, a + 1); ++p) {
      const double cap = c_entry(s, a, p);
      if (cap == 0.0) continue;
      if (!sandwich) {
        const cplx xv = Xe[(int64_t)p * nx + b];
        re += cap * xv.x;
        im += cap * xv.y;
      } else {
        for (int q = max(0, b - 1); q <= min(nx - 1, b + 1); ++q) {
          const double w = cap * c_entry(s, q, b);
          if (w == 0.0) continue;
          const cplx xv = Xe[(int64_t)p * nx + q];
          re += w * xv.x;
          im += w * xv.y;
        }
      }
    }
    row[b] = make_double2(sign * re, sign * im);
  }
}

// out[x] (+)= sum_b P[x][b] conj(Q[x][b]) for x < nx: the diagonal of P Q^H;
// with diag_src != nullptr also diagG[x] = diag_src[x][x].
__global__ void __launch_bounds__(128) k_rgf_diag(RgfSlice s, const cplx* __restrict__ P,
                                                 const cplx* __restrict__ Q, int64_t stride,
                                                 cplx* __restrict__ out, int64_t ostride, int accumulate,
                                                 const cplx* __restrict__ diag_src, cplx* __restrict__ diagG) {
  const int x = blockIdx.x, e = blockIdx.y, nx = s.nx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double sr[4], si[4];
  double re = 0.0, im = 0.0;
  if (P) {
    const cplx* pr = P + (int64_t)e * stride + (int64_t)x * nx;
    const cplx* qr = Q + (int64_t)e * stride + (int64_t)x * nx;
    for (int b = threadIdx.x; b < nx; b += blockDim.x) {
      const cplx p = pr[b], q = qr[b];
      re += p.x * q.x + p.y * q.y;
      im += p.y * q.x - p.x * q.y;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  if (lane == 0) { sr[warp] = re; si[warp] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    re = sr[0] + sr[1] + sr[2] + sr[3];
    im = si[0] + si[1] + si[2] + si[3];
    cplx* o = out + (int64_t)e * ostride + x;
    if (P) {
      if (accumulate) *o = make_double2(o->x + re, o->y + im);
      else *o = make_double2(re, im);
    }
    if (diag_src) diagG[(int64_t)e * ostride + x] = diag_src[(int64_t)e * stride + (int64_t)x * nx + x];
  }
}

// Sigma< of a contact: out = -f (sig - sig^H) = i f Gamma
__global__ void k_rgf_lesser(const cplx* __restrict__ sig, int nx, double f, cplx* __restrict__ out) {
  const int a = blockIdx.x, e = blockIdx.y;
  const cplx* se = sig + (int64_t)e * nx * nx;
  for (int b = threadIdx.x; b < nx; b += blockDim.x) {
    const cplx u = se[(int64_t)a * nx + b], v = se[(int64_t)b * nx + a];
    out[((int64_t)e * nx + a) * nx + b] = make_double2(-f * (u.x - v.x), -f * (u.y + v.y));
  }
}

void launch_rgf_lesser(const cplx* sig, int nx, double f, cplx* out, int nE, cudaStream_t st) {
  k_rgf_lesser<<<dim3(nx, nE), 128, 0, st>>>(sig, nx, f, out);
}

void launch_rgf_block(const RgfSlice& s, int y, const cplx* X, int64_t xstride, cplx* M, int64_t mstride,
                      int nE, cudaStream_t st) {
  k_rgf_block<<<dim3(s.nx, nE), 256, 0, st>>>(s, y, X, xstride, M, mstride);
}

void launch_rgf_cprod(const RgfSlice& s, const cplx* X, int64_t xstride, cplx* W, int64_t wstride,
                      double sign, int sandwich, int nE, cudaStream_t st) {
  k_rgf_cprod<<<dim3(s.nx, nE), 256, 0, st>>>(s, X, xstride, W, wstride, sign, sandwich);
}

void launch_rgf_diag(const RgfSlice& s, const cplx* P, const cplx* Q, int64_t stride, cplx* out,
                     int64_t ostride, int accumulate, const cplx* diag_src, cplx* diagG, int nE,
                     cudaStream_t st) {
  k_rgf_diag<<<dim3(s.nx, nE), 128, 0, st>>>(s, P, Q, stride, out, ostride, accumulate, diag_src, diagG);
}

}  // namespace findgb
