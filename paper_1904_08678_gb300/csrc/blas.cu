// BLAS-1 kernels and the device-side Arnoldi/Givens bookkeeping of the Krylov
// solvers (Sec. 2.1: MR, GMRES, FGMRES).  Fields are batches [nrhs][n] of
// complex numbers; every per-rhs scalar stays in device memory so the solver
// loops issue no host round trip except their stopping tests.
// Reductions are two-stage with fixed block counts and fixed summation trees:
// results are bitwise reproducible run to run.
#include <algorithm>

#include <cooperative_groups.h>

#include "kernels.h"

namespace wcmg {

constexpr int RED_T = 256;
// Blocks along the vector of a two-stage reduction: about 8 elements per thread
// for long vectors, but never fewer CTAs (over all `others` = rhs x chunks) than
// ~4 per SM while every thread still has an element: short coarse vectors are
// spread over the GPU instead of a dozen CTAs.  At most 608 (partial buffers).
static inline int red_blocks(long long n, long long others = 1) {
  const long long per8 = (n + 8 * RED_T - 1) / (8 * RED_T);
  const long long per1 = (n + RED_T - 1) / RED_T;
  const long long want = (4 * 152 + others - 1) / others;
  long long b = std::min(std::max(per8, want), per1);
  return (int)(b < 1 ? 1 : (b > 608 ? 608 : b));
}

template <typename A, typename B>
__global__ void k_convert(cplx<B>* __restrict__ out, const cplx<A>* __restrict__ in, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = from_c64<B>(to_c64(in[i]));
}
template <typename A, typename B>
void launch_convert(cplx<B>* out, const cplx<A>* in, long long n, cudaStream_t st) {
  k_convert<A, B><<<nblk(n, 256), 256, 0, st>>>(out, in, n);
  WCMG_LAUNCH_CHECK();
}

// ---- dot / norm ----
template <typename R>
__global__ void __launch_bounds__(RED_T) k_dot_partial(double2* __restrict__ partial, const cplx<R>* __restrict__ a,
                                                       const cplx<R>* __restrict__ b, long long n) {
  __shared__ double2 scratch[RED_T / 32];
  __shared__ double2 red[1];
  const int r = blockIdx.y;
  a += (long long)r * n;
  b += (long long)r * n;
  cplx<R> acc = czero<R>();
  for (long long i = blockIdx.x * (long long)RED_T + threadIdx.x; i < n; i += (long long)gridDim.x * RED_T)
    cjmac(acc, a[i], b[i]);
  const R v[2] = {acc.x, acc.y};
  double* sd = reinterpret_cast<double*>(scratch);
  double* rd = reinterpret_cast<double*>(red);
  block_sum_mixed<R, 2>(v, sd, rd);
  if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = make_double2(rd[0], rd[1]);
}
template <typename R>
__global__ void __launch_bounds__(RED_T) k_norm_partial(double* __restrict__ partial, const cplx<R>* __restrict__ a,
                                                        long long n) {
  __shared__ double scratch[RED_T / 32];
  __shared__ double red[1];
  const int r = blockIdx.y;
  a += (long long)r * n;
  R acc = 0;
  for (long long i = blockIdx.x * (long long)RED_T + threadIdx.x; i < n; i += (long long)gridDim.x * RED_T)
    acc += cnorm2(a[i]);
  const R v[1] = {acc};
  block_sum_mixed<R, 1>(v, scratch, red);
  if (threadIdx.x == 0) partial[(long long)r * gridDim.x + blockIdx.x] = red[0];
}
// out[r * ldo + i] = sum_{b < count} partial[r * pr + i * pi + b]  (grid: r = x, i = y)
// lim (nullable): rows i >= *lim + ladd are skipped (a device-side Arnoldi step count).
template <typename T>
__global__ void __launch_bounds__(RED_T) k_final(T* __restrict__ out, const T* __restrict__ partial, int count,
                                                 long long pr, long long pi, int ldo, const int* __restrict__ lim = nullptr,
                                                 int ladd = 0) {
  __shared__ T scratch[RED_T / 32];
  __shared__ T red[1];
  const int r = blockIdx.x, i = blockIdx.y;
  if (lim && i >= *lim + ladd) return;  // uniform per block
  const T* p = partial + r * pr + i * pi;
  T acc;
  memset(&acc, 0, sizeof(T));
  for (int b = threadIdx.x; b < count; b += RED_T) acc += p[b];
  block_sum_many<T>(&acc, 1, scratch, red);
  if (threadIdx.x == 0) out[(long long)r * ldo + i] = red[0];
}

template <typename R>
void launch_dot(double2* out, const cplx<R>* a, const cplx<R>* b, long long n, int nrhs, double2* partial,
                cudaStream_t st) {
  const int nb = red_blocks(n, nrhs);
  k_dot_partial<R><<<dim3(nb, nrhs), RED_T, 0, st>>>(partial, a, b, n);
  k_final<double2><<<dim3(nrhs, 1), RED_T, 0, st>>>(out, partial, nb, nb, 0, 1);
  ++launch_counter();
  WCMG_LAUNCH_CHECK();
}
template <typename R>
void launch_norm2(double* out, const cplx<R>* a, long long n, int nrhs, double* partial, cudaStream_t st) {
  const int nb = red_blocks(n, nrhs);
  k_norm_partial<R><<<dim3(nb, nrhs), RED_T, 0, st>>>(partial, a, n);
  k_final<double><<<dim3(nrhs, 1), RED_T, 0, st>>>(out, partial, nb, nb, 0, 1);
  ++launch_counter();
  WCMG_LAUNCH_CHECK();
}

// ---- multi-dot against a Krylov basis (chunks of 8 basis vectors) ----
constexpr int MD_K = 8;
template <typename R>
__global__ void __launch_bounds__(RED_T) k_multidot_partial(double2* __restrict__ partial,
                                                            const cplx<R>* __restrict__ basis, long long bstride,
                                                            int k, const cplx<R>* __restrict__ w, long long n,
                                                            int kpad, const int* __restrict__ kdev, int kadd,
                                                            int vec2) {
  __shared__ double2 scratch[(RED_T / 32) * MD_K];
  const int r = blockIdx.y, i0 = blockIdx.z * MD_K;
  if (kdev) k = *kdev + kadd;
  if (i0 >= k) return;  // uniform per block
  const long long off = (long long)r * n;
  cplx<R> acc[MD_K];
#pragma unroll
  for (int q = 0; q < MD_K; ++q) acc[q] = czero<R>();
  if constexpr (sizeof(R) == 4) {
    if (vec2) {  // two complex entries per 16-byte load (n, bstride even; 16-byte aligned fields)
      const float4* w4 = reinterpret_cast<const float4*>(w + off);
      const long long n2 = n >> 1;
      for (long long e = blockIdx.x * (long long)RED_T + threadIdx.x; e < n2; e += (long long)gridDim.x * RED_T) {
        const float4 x = w4[e];
#pragma unroll
        for (int q = 0; q < MD_K; ++q)
          if (i0 + q < k) {
            const float4 v = reinterpret_cast<const float4*>(basis + (i0 + q) * bstride + off)[e];
            cjmac(acc[q], make_float2(v.x, v.y), make_float2(x.x, x.y));
            cjmac(acc[q], make_float2(v.z, v.w), make_float2(x.z, x.w));
          }
      }
      vec2 = -1;  // done
    }
  }
  if (vec2 >= 0)
    for (long long e = blockIdx.x * (long long)RED_T + threadIdx.x; e < n; e += (long long)gridDim.x * RED_T) {
      const cplx<R> x = w[off + e];
#pragma unroll
      for (int q = 0; q < MD_K; ++q)
        if (i0 + q < k) cjmac(acc[q], basis[(i0 + q) * bstride + off + e], x);
    }
  // warp sums in the working precision (one transposing butterfly for the 8 values),
  // then FP64 across the warps of the CTA and across CTAs
  static_assert(MD_K == 8, "transposing warp reduction of 8 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum8_transposed(acc, lane);
  if ((lane & 3) == 0) scratch[warp * MD_K + warp_sum8_index(lane)] = to_c64(acc[0]);
  __syncthreads();
  if (threadIdx.x < MD_K && i0 + threadIdx.x < k) {
    double2 t = scratch[threadIdx.x];
    for (int w = 1; w < RED_T / 32; ++w) t += scratch[w * MD_K + threadIdx.x];
    partial[((long long)r * kpad + i0 + threadIdx.x) * gridDim.x + blockIdx.x] = t;
  }
}
// k basis vectors; with kdev the count is *kdev + kadd (<= k) read on the device.
template <typename R>
void launch_multidot(double2* out, const cplx<R>* basis, long long bstride, int k, int ldo, const cplx<R>* w,
                     long long n, int nrhs, double2* partial, cudaStream_t st, const int* kdev, int kadd) {
  const int nchunk = (k + MD_K - 1) / MD_K, kpad = nchunk * MD_K;
  const int nb = red_blocks(n, nrhs);  // independent of k: a captured graph sums in the same order
  const int vec2 = sizeof(R) == 4 && n % 2 == 0 && bstride % 2 == 0 && reinterpret_cast<uintptr_t>(basis) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(w) % 16 == 0;
  k_multidot_partial<R><<<dim3(nb, nrhs, nchunk), RED_T, 0, st>>>(partial, basis, bstride, k, w, n, kpad, kdev, kadd,
                                                                  vec2);
  k_final<double2><<<dim3(nrhs, k), RED_T, 0, st>>>(out, partial, nb, (long long)kpad * nb, nb, ldo, kdev, kadd);
  ++launch_counter();
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_multiaxpy(cplx<R>* __restrict__ w, const cplx<R>* __restrict__ basis, long long bstride, int k,
                           const double2* __restrict__ coef, int ldc, double sign, long long n,
                           const int* __restrict__ kdev, int kadd) {
  __shared__ cplx<R> cf[80];  // k <= 65 (restart <= 64)
  const int r = blockIdx.y;
  if (kdev) k = min(*kdev + kadd, k);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double2 c = coef[(long long)r * ldc + i];
    cf[i] = cmk(R(sign * c.x), R(sign * c.y));
  }
  __syncthreads();
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const long long off = (long long)r * n + e;
  cplx<R> acc = w[off];
  for (int i = 0; i < k; ++i) cmac(acc, cf[i], basis[i * bstride + off]);
  w[off] = acc;
}
template <typename R>
void launch_multiaxpy(cplx<R>* w, const cplx<R>* basis, long long bstride, int k, const double2* coef, int ldc,
                      double sign, long long n, int nrhs, cudaStream_t st, const int* kdev, int kadd) {
  if (k <= 0) return;
  if (k > 80) throw Error(-1, "multiaxpy supports k <= 80");
  k_multiaxpy<R><<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(w, basis, bstride, k, coef, ldc, sign, n, kdev, kadd);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_axpby(cplx<R>* __restrict__ y, R a, const cplx<R>* __restrict__ x, R b, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}
template <typename R>
void launch_axpby(cplx<R>* y, double a, const cplx<R>* x, double b, long long n, int nrhs, cudaStream_t st) {
  const long long N = n * nrhs;
  k_axpby<R><<<nblk(N, 256), 256, 0, st>>>(y, (R)a, x, (R)b, N);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_scale_dev(cplx<R>* __restrict__ y, const cplx<R>* __restrict__ x, const double* __restrict__ s,
                            int inv_sqrt, long long n, const int* __restrict__ ydev, int yadd, long long ystride) {
  __shared__ R f_s;
  const int r = blockIdx.y;
  if (ydev) y += (long long)(*ydev + yadd) * ystride;
  if (threadIdx.x == 0) {
    double f = s[r];
    if (inv_sqrt) f = f > 0.0 ? 1.0 / sqrt(f) : 0.0;
    f_s = (R)f;
  }
  __syncthreads();
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  y[(long long)r * n + e] = f_s * x[(long long)r * n + e];
}
template <typename R>
void launch_scale_dev(cplx<R>* y, const cplx<R>* x, const double* s, int inv_sqrt, long long n, int nrhs,
                      cudaStream_t st, const int* ydev, int yadd, long long ystride) {
  k_scale_dev<R><<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(y, x, s, inv_sqrt, n, ydev, yadd, ystride);
  WCMG_LAUNCH_CHECK();
}

// The step reads the residual from rin and writes the new one to r (rin = r in place;
// the first step reads b itself).  X_ZERO: x is known to be 0 (first step: not read);
// R_NEXT = false: the new r is not needed (last step: not written).  Same arithmetic in
// every variant.
template <typename R, bool X_ZERO, bool R_NEXT>
__global__ void k_mr_update(cplx<R>* __restrict__ x, cplx<R>* r, const cplx<R>* rin, const cplx<R>* __restrict__ p,
                            const double2* __restrict__ pr, const double* __restrict__ pp, long long n) {
  __shared__ cplx<R> a_s;
  const int q = blockIdx.y;
  if (threadIdx.x == 0) {
    const double d = pp[q];
    a_s = d != 0.0 ? cmk((R)(pr[q].x / d), (R)(pr[q].y / d)) : czero<R>();
  }
  __syncthreads();
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const cplx<R> a = a_s;
  const long long o = (long long)q * n + e;
  const cplx<R> rv = rin[o];
  cplx<R> xv = X_ZERO ? czero<R>() : x[o];
  cmac(xv, a, rv);
  x[o] = xv;
  if (R_NEXT) r[o] = rv - cmul(a, p[o]);
}
template <typename R>
void launch_mr_update(cplx<R>* x, cplx<R>* r, const cplx<R>* p, const double2* pr, const double* pp, long long n,
                      int nrhs, cudaStream_t st, bool x_zero, bool r_next, const cplx<R>* rin) {
  const dim3 grid(nblk(n, 256), nrhs);
  if (!rin) rin = r;
  if (x_zero && r_next) k_mr_update<R, true, true><<<grid, 256, 0, st>>>(x, r, rin, p, pr, pp, n);
  else if (x_zero) k_mr_update<R, true, false><<<grid, 256, 0, st>>>(x, r, rin, p, pr, pp, n);
  else if (r_next) k_mr_update<R, false, true><<<grid, 256, 0, st>>>(x, r, rin, p, pr, pp, n);
  else k_mr_update<R, false, false><<<grid, 256, 0, st>>>(x, r, rin, p, pr, pp, n);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_mask_rhs(cplx<R>* __restrict__ x, const int* __restrict__ mask, long long n) {
  const int r = blockIdx.y;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < n && mask[r]) x[(long long)r * n + e] = czero<R>();
}
template <typename R>
void launch_mask_rhs(cplx<R>* x, const int* mask, long long n, int nrhs, cudaStream_t st) {
  k_mask_rhs<R><<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(x, mask, n);
  WCMG_LAUNCH_CHECK();
}

// dst[o * dmul + i] = src[o * smul + i], o = *idx (0 when idx is null): the copy of
// one Krylov basis slot selected on the device.
template <typename R>
__global__ void k_copy_idx(cplx<R>* __restrict__ dst, const cplx<R>* __restrict__ src, long long n,
                           const int* __restrict__ idx, long long dmul, long long smul) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long o = idx ? *idx : 0;
  dst[o * dmul + i] = src[o * smul + i];
}
template <typename R>
void launch_copy_idx(cplx<R>* dst, const cplx<R>* src, long long n, const int* idx, long long dmul, long long smul,
                     cudaStream_t st) {
  if (n <= 0) return;
  k_copy_idx<R><<<nblk(n, 256), 256, 0, st>>>(dst, src, n, idx, dmul, smul);
  WCMG_LAUNCH_CHECK();
}
__global__ void k_fill_int(int* x, int v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = v;
}
void launch_fill_int(int* x, int v, int n, cudaStream_t st) {
  if (n <= 0) return;
  k_fill_int<<<nblk(n, 256), 256, 0, st>>>(x, v, n);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_fill_zero(cplx<R>* x, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) x[i] = czero<R>();
}
template <typename R>
void launch_fill_zero(cplx<R>* x, long long n, cudaStream_t st) {
  if (n <= 0) return;
  k_fill_zero<R><<<nblk(n, 256), 256, 0, st>>>(x, n);
  WCMG_LAUNCH_CHECK();
}

// ---- (F)GMRES bookkeeping (K8), one thread per rhs, FP64 ----
// Complex Givens rotation G = [[c, s], [-conj(s), c]], c real, with
// G [a, b]^T = [rho, 0]^T.
__device__ void givens(double2 a, double2 b, double& c, double2& s, double2& rho) {
  const double aa = sqrt(cnorm2(a));
  if (aa == 0.0) { c = 0.0; s = make_double2(1, 0); rho = b; return; }
  const double r = sqrt(cnorm2(a) + cnorm2(b));
  const double2 ph = make_double2(a.x / aa, a.y / aa);
  c = aa / r;
  s = (1.0 / r) * cmul(ph, conjg(b));
  rho = r * ph;
}

__global__ void k_gmres_start(GmresState S, const double* __restrict__ nrm2, double tol, int nrhs,
                              double* __restrict__ inv_beta) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double beta = sqrt(nrm2[r]);
  const int m = S.m;
  for (int i = 0; i <= m; ++i) S.g[(long long)r * (m + 1) + i] = make_double2(0, 0);
  S.g[(long long)r * (m + 1)] = make_double2(beta, 0);
  S.resid[r] = beta;
  S.jdone[r] = 0;
  const bool go = !S.done[r] && beta > tol * S.bnorm[r] && beta > 0.0;
  S.active[r] = go ? 1 : 0;
  inv_beta[r] = go ? 1.0 / beta : 0.0;
}

// Column j of the Hessenberg matrix of rhs r: h_col[0..j] (both CGS passes summed)
// and ||w||^2; the earlier rotations, a new complex Givens rotation and the
// recurrence residual; returns 1 / ||w|| (0 if ||w|| = 0).
__device__ double gmres_column(GmresState S, int r, int j, const double2* hcol, double hn2, double tol,
                               int final_done) {
  const int m = S.m;
  double2* H = S.H + (long long)r * (m + 1) * m;
  double* cs = S.cs + (long long)r * m;
  double2* sn = S.sn + (long long)r * m;
  double2* g = S.g + (long long)r * (m + 1);
  for (int i = 0; i <= j; ++i) H[i * m + j] = hcol[i];
  const double h = sqrt(hn2);
  H[(j + 1) * m + j] = make_double2(h, 0);
  for (int i = 0; i < j; ++i) {
    const double2 a = H[i * m + j], b = H[(i + 1) * m + j];
    H[i * m + j] = cs[i] * a + cmul(sn[i], b);
    H[(i + 1) * m + j] = cs[i] * b - cmul(conjg(sn[i]), a);
  }
  double c; double2 s, rho;
  givens(H[j * m + j], H[(j + 1) * m + j], c, s, rho);
  cs[j] = c; sn[j] = s;
  H[j * m + j] = rho;
  H[(j + 1) * m + j] = make_double2(0, 0);
  const double2 gj = g[j];
  g[j + 1] = -cmul(conjg(s), gj);
  g[j] = c * gj;
  const double res = sqrt(cnorm2(g[j + 1]));
  S.resid[r] = res;
  S.jdone[r] = j + 1;
  if (res <= tol * S.bnorm[r]) {
    S.active[r] = 0;
    if (final_done) S.done[r] = 1;
  }
  return h > 0.0 ? 1.0 / h : 0.0;
}

__global__ void k_gmres_step(GmresState S, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                             const double* __restrict__ hnorm2, double tol, int final_done, int nrhs,
                             double* __restrict__ inv_h, const int* __restrict__ jdev) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  if (jdev) j = *jdev;
  const int m = S.m;
  if (!S.active[r]) { inv_h[r] = 0.0; return; }
  double2 hcol[65];
  for (int i = 0; i <= j; ++i) hcol[i] = h1[(long long)r * (m + 1) + i] + h2[(long long)r * (m + 1) + i];
  inv_h[r] = gmres_column(S, r, j, hcol, hnorm2[r], tol, final_done);
}

// ---- fused Arnoldi step for short vectors (one rhs) ----
// Everything of one (F)GMRES Arnoldi step after the operator application, for
// vectors short enough that a single thread-block cluster streams them from L2:
// both classical Gram-Schmidt passes h1 = V^dag w, w -= V h1, h2 = V^dag w,
// w -= V h2, the norm ||w||^2, the Givens update of Hessenberg column j and
// V_{j+1} = w / ||w||.  CTA c of the C-CTA cluster owns a contiguous range of the
// vector; its partial sums (warp sums in the working precision, FP64 across
// warps) are exchanged through distributed shared memory, and every CTA adds the C
// partials in the same order, so all CTAs hold identical coefficients.  One
// launch replaces ten (three two-stage reductions, two updates, Givens, scaling).
constexpr int AC_T = 256, AC_MAXK = 65;

template <typename R>
__device__ __forceinline__ void ac_reduce8(cplx<R> (&acc)[8], double2* __restrict__ scr, double2* __restrict__ out,
                                           int i0, int k) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_sum8_transposed(acc, lane);
  if ((lane & 3) == 0) scr[warp * 8 + warp_sum8_index(lane)] = to_c64(acc[0]);
  __syncthreads();
  if (threadIdx.x < 8 && i0 + threadIdx.x < k) {
    double2 t = scr[threadIdx.x];
    for (int w = 1; w < AC_T / 32; ++w) t += scr[w * 8 + threadIdx.x];
    out[i0 + threadIdx.x] = t;
  }
  __syncthreads();
}

template <typename R>
__global__ void __launch_bounds__(AC_T) k_arnoldi_cluster(cplx<R>* __restrict__ Vb, long long bstride,
                                                          cplx<R>* __restrict__ w, long long n, GmresState S, int j,
                                                          const int* __restrict__ jdev, double tol, int final_done) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  __shared__ double2 pA[AC_MAXK], pB[AC_MAXK];  // this CTA's partial sums (read by the whole cluster)
  __shared__ double pN;
  __shared__ double2 h1s[AC_MAXK], hcol[AC_MAXK];
  __shared__ double2 scr[(AC_T / 32) * 8];
  __shared__ double dscr[AC_T / 32];
  if (jdev) j = *jdev;
  const int k = j + 1;
  const bool act = S.active[0] != 0;  // before this step (CTA 0 may change it below)
  const long long per = (n + C - 1) / C;
  const long long e0 = (long long)crank * per, e1 = e0 + per < n ? e0 + per : n;
  // pass 1: <V_i, w>
  for (int i0 = 0; i0 < k; i0 += 8) {
    cplx<R> acc[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) acc[g] = czero<R>();
    for (long long e = e0 + threadIdx.x; e < e1; e += AC_T) {
      const cplx<R> x = w[e];
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (i0 + g < k) cjmac(acc[g], Vb[(i0 + g) * bstride + e], x);
    }
    ac_reduce8<R>(acc, scr, pA, i0, k);
  }
  cl.sync();
  for (int i = threadIdx.x; i < k; i += AC_T) {
    double2 t = make_double2(0, 0);
    for (int c = 0; c < C; ++c) t += cl.map_shared_rank(pA, c)[i];
    h1s[i] = t;
  }
  __syncthreads();
  // w -= V h1, then pass 2: <V_i, w>  (each thread revisits only its own elements)
  for (long long e = e0 + threadIdx.x; e < e1; e += AC_T) {
    cplx<R> x = w[e];
    for (int i = 0; i < k; ++i) {
      const double2 h = h1s[i];
      cnmac(x, cmk(R(h.x), R(h.y)), Vb[i * bstride + e]);
    }
    w[e] = x;
  }
  for (int i0 = 0; i0 < k; i0 += 8) {
    cplx<R> acc[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) acc[g] = czero<R>();
    for (long long e = e0 + threadIdx.x; e < e1; e += AC_T) {
      const cplx<R> x = w[e];
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (i0 + g < k) cjmac(acc[g], Vb[(i0 + g) * bstride + e], x);
    }
    ac_reduce8<R>(acc, scr, pB, i0, k);
  }
  cl.sync();
  for (int i = threadIdx.x; i < k; i += AC_T) {
    double2 t = make_double2(0, 0);
    for (int c = 0; c < C; ++c) t += cl.map_shared_rank(pB, c)[i];
    hcol[i] = h1s[i] + t;
    h1s[i] = t;  // h2
  }
  __syncthreads();
  // w -= V h2 and ||w||^2
  R nn = 0;
  for (long long e = e0 + threadIdx.x; e < e1; e += AC_T) {
    cplx<R> x = w[e];
    for (int i = 0; i < k; ++i) {
      const double2 h = h1s[i];
      cnmac(x, cmk(R(h.x), R(h.y)), Vb[i * bstride + e]);
    }
    w[e] = x;
    nn += cnorm2(x);
  }
  {
    const R v[1] = {nn};
    double red[1];
    block_sum_mixed<R, 1>(v, dscr, red);
    if (threadIdx.x == 0) pN = red[0];
  }
  cl.sync();
  double hn2 = 0.0;
  for (int c = 0; c < C; ++c) hn2 += *cl.map_shared_rank(&pN, c);
  // V_{j+1} = w / ||w|| and, on one thread, the Givens update of column j
  const double h = sqrt(hn2);
  const R inv = (R)(act && h > 0.0 ? 1.0 / h : 0.0);
  cplx<R>* vn = Vb + (long long)(j + 1) * bstride;
  for (long long e = e0 + threadIdx.x; e < e1; e += AC_T) vn[e] = inv * w[e];
  if (crank == 0 && threadIdx.x == 0 && act) gmres_column(S, 0, j, hcol, hn2, tol, final_done);
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

static int arnoldi_cluster_size() {
  static int cached = -1;
  if (cached >= 0) return cached;
  cached = 0;
  for (int C : {16, 8}) {
    auto kern = k_arnoldi_cluster<float>;
    if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(AC_T);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0) {
      cached = C;
      break;
    }
    cudaGetLastError();
  }
  return cached;
}

// The 16-CTA cluster reads the basis through 16 SMs only: it beats the seven
// whole-GPU launches it replaces for short vectors (the coarsest levels: 10^4 - 4 x 10^4
// entries) but not for fine-level ones (a 16^4 lattice, 7.9 x 10^5 entries: 300 us per
// step against about 60 us), so it takes vectors of at most 2^17 entries.
bool arnoldi_fused_ok(long long n, int nrhs, int m) {
  return nrhs == 1 && m + 1 <= AC_MAXK && n <= (1LL << 17) && arnoldi_cluster_size() > 0;
}

template <typename R>
void launch_arnoldi_fused(cplx<R>* Vb, long long bstride, cplx<R>* w, long long n, const GmresState& S, int j,
                          const int* jdev, double tol, int final_done, cudaStream_t st) {
  const int C = arnoldi_cluster_size();
  if (C <= 0) throw Error(-1, "no thread-block cluster available for the fused Arnoldi step");
  auto kern = k_arnoldi_cluster<R>;
  if (C > 8) WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(AC_T);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  WCMG_CUDA(cudaLaunchKernelEx(&cfg, kern, Vb, bstride, w, n, S, j, jdev, tol, final_done));
  WCMG_LAUNCH_CHECK();
}
template void launch_arnoldi_fused<float>(float2*, long long, float2*, long long, const GmresState&, int, const int*,
                                          double, int, cudaStream_t);
template void launch_arnoldi_fused<double>(double2*, long long, double2*, long long, const GmresState&, int,
                                           const int*, double, int, cudaStream_t);

__global__ void k_gmres_solve_y(GmresState S, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const int m = S.m, jd = S.jdone[r];
  const double2* H = S.H + (long long)r * (m + 1) * m;
  const double2* g = S.g + (long long)r * (m + 1);
  double2* y = S.y + (long long)r * m;
  for (int i = m - 1; i >= jd; --i) y[i] = make_double2(0, 0);
  for (int i = jd - 1; i >= 0; --i) {
    double2 t = g[i];
    for (int k = i + 1; k < jd; ++k) t -= cmul(H[i * m + k], y[k]);
    const double2 d = H[i * m + i];
    const double dd = cnorm2(d);
    y[i] = dd > 0.0 ? (1.0 / dd) * cjmul(d, t) : make_double2(0, 0);
  }
}

__global__ void k_gmres_mark_done(GmresState S, const double* __restrict__ nrm2, double tol, int nrhs) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const double lim = tol * S.bnorm[r];
  if (sqrt(nrm2[r]) <= lim) S.done[r] = 1;
}

void launch_gmres_start(const GmresState& s, const double* nrm2, double tol, int nrhs, double* inv_beta,
                        cudaStream_t st) {
  k_gmres_start<<<nblk(nrhs, 64), 64, 0, st>>>(s, nrm2, tol, nrhs, inv_beta);
  WCMG_LAUNCH_CHECK();
}
void launch_gmres_step(const GmresState& s, int j, const double2* h1, const double2* h2, const double* hnorm2,
                       double tol, int final_done, int nrhs, double* inv_h, cudaStream_t st, const int* jdev) {
  k_gmres_step<<<nblk(nrhs, 64), 64, 0, st>>>(s, j, h1, h2, hnorm2, tol, final_done, nrhs, inv_h, jdev);
  WCMG_LAUNCH_CHECK();
}
void launch_gmres_solve_y(const GmresState& s, int nrhs, cudaStream_t st) {
  k_gmres_solve_y<<<nblk(nrhs, 64), 64, 0, st>>>(s, nrhs);
  WCMG_LAUNCH_CHECK();
}
void launch_gmres_mark_done(const GmresState& s, const double* nrm2, double tol, int nrhs, cudaStream_t st) {
  k_gmres_mark_done<<<nblk(nrhs, 64), 64, 0, st>>>(s, nrm2, tol, nrhs);
  WCMG_LAUNCH_CHECK();
}

// ---- counter-based Gaussian fields (the generator of the seeded inputs) ----
// Element j of field i (stream stream0 + i): the counter c = seed * 0x9E3779B97F4A7C15
// + stream * 0xD1B54A32D192ED03 + k (mod 2^64) for k = 2j, 2j+1 goes through the
// SplitMix64 finaliser (Steele, Lea, Flood, OOPSLA 2014); u = (out >> 11) 2^-53 exactly;
// Box-Muller: re = sqrt(-2 log(1 - u_2j)) cos(2 pi u_2j+1), im = the same with sin.  The
// transform runs in FP32 (1 - u is formed exactly in FP64 first, so it never rounds to
// 0): FP64 transcendentals on this part would cost more than copying the fields in.
__device__ __forceinline__ double counter_uniform(unsigned long long base, unsigned long long k) {
  unsigned long long z = base + k;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * 0x1.0p-53;
}
__global__ void k_counter_gaussian(double2* __restrict__ out, long long n, unsigned long long seed,
                                   unsigned long long stream0) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const unsigned long long stream = stream0 + blockIdx.y;
  const unsigned long long base = seed * 0x9E3779B97F4A7C15ULL + stream * 0xD1B54A32D192ED03ULL;
  const double u1 = counter_uniform(base, 2ULL * j), u2 = counter_uniform(base, 2ULL * j + 1);
  const float r = sqrtf(-2.0f * logf((float)(1.0 - u1)));
  float sn, cs;
  sincospif((float)(2.0 * u2), &sn, &cs);
  out[(long long)blockIdx.y * n + j] = make_double2((double)(r * cs), (double)(r * sn));
}
void launch_counter_gaussian(double2* out, long long n, int nfields, unsigned long long seed,
                             unsigned long long stream0, cudaStream_t st) {
  k_counter_gaussian<<<dim3(nblk(n, 256), nfields), 256, 0, st>>>(out, n, seed, stream0);
  WCMG_LAUNCH_CHECK();
}

#define WCMG_INST(R)                                                                                             \
  template void launch_dot<R>(double2*, const cplx<R>*, const cplx<R>*, long long, int, double2*, cudaStream_t); \
  template void launch_norm2<R>(double*, const cplx<R>*, long long, int, double*, cudaStream_t);                 \
  template void launch_multidot<R>(double2*, const cplx<R>*, long long, int, int, const cplx<R>*, long long, int, \
                                   double2*, cudaStream_t, const int*, int);                                     \
  template void launch_multiaxpy<R>(cplx<R>*, const cplx<R>*, long long, int, const double2*, int, double,       \
                                    long long, int, cudaStream_t, const int*, int);                              \
  template void launch_copy_idx<R>(cplx<R>*, const cplx<R>*, long long, const int*, long long, long long,        \
                                   cudaStream_t);                                                                \
  template void launch_axpby<R>(cplx<R>*, double, const cplx<R>*, double, long long, int, cudaStream_t);         \
  template void launch_scale_dev<R>(cplx<R>*, const cplx<R>*, const double*, int, long long, int, cudaStream_t,  \
                                    const int*, int, long long);                                                 \
  template void launch_mr_update<R>(cplx<R>*, cplx<R>*, const cplx<R>*, const double2*, const double*, long long, \
                                    int, cudaStream_t, bool, bool, const cplx<R>*);                              \
  template void launch_mask_rhs<R>(cplx<R>*, const int*, long long, int, cudaStream_t);                          \
  template void launch_fill_zero<R>(cplx<R>*, long long, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST
template void launch_convert<double, float>(float2*, const double2*, long long, cudaStream_t);
template void launch_convert<float, double>(double2*, const float2*, long long, cudaStream_t);
template void launch_convert<double, double>(double2*, const double2*, long long, cudaStream_t);
template void launch_convert<float, float>(float2*, const float2*, long long, cudaStream_t);

}  // namespace wcmg

namespace wcmg {
__global__ void k_sqrt_inplace(double* x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = sqrt(x[i]);
}
void launch_sqrt_inplace(double* x, int n, cudaStream_t st) {
  k_sqrt_inplace<<<nblk(n, 64), 64, 0, st>>>(x, n);
  WCMG_LAUNCH_CHECK();
}
}  // namespace wcmg
