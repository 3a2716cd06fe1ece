// Schwarz alternating procedure (SAP) smoother pieces (Sec. 4 names SAP as the usual
// smoother on every level).  The Schwarz blocks are the level's aggregates, which the
// storage order keeps contiguous: block B holds sites [B |B|, (B+1) |B|).  Blocks are
// coloured by the parity of their coarse-lattice coordinates; a colour pass solves
// D_B e = r on every block of one colour with block-local minimal-residual steps, each
// block with its own step length.
#include "kernels.h"

namespace wcmg {

// Offset of element e (0 <= e < |B| nc) of block B in one rhs: fine fields are
// component-major [nc][V], coarse fields site-major [V][nc].
__device__ __forceinline__ long long block_elem(int B, int e, int bvol, int nc, int V, bool fine) {
  if (fine) {
    const int k = e / bvol, i = e - k * bvol;
    return (long long)k * V + (long long)B * bvol + i;
  }
  return (long long)B * bvol * nc + e;
}

// r = colour(B(site)) == c ? b - Dx : 0   (Dx null: the x = 0 case, r = b there)
template <typename R>
__global__ void k_sap_residual(cplx<R>* __restrict__ r, const cplx<R>* __restrict__ b,
                               const cplx<R>* __restrict__ Dx, const unsigned char* __restrict__ colour, int c,
                               int V, int nc, int bvol, bool fine, long long n) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const long long o = (long long)blockIdx.y * n + e;
  const int site = fine ? (int)(e % V) : (int)(e / nc);
  cplx<R> v = czero<R>();
  if (colour[site / bvol] == c) v = Dx ? b[o] - Dx[o] : b[o];
  r[o] = v;
}
template <typename R>
void launch_sap_residual(cplx<R>* r, const cplx<R>* b, const cplx<R>* Dx, const unsigned char* colour, int c, int V,
                         int nc, int bvol, bool fine, int nrhs, cudaStream_t st) {
  const long long n = (long long)V * nc;
  k_sap_residual<R><<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(r, b, Dx, colour, c, V, nc, bvol, fine, n);
  WCMG_LAUNCH_CHECK();
}

// One block-local MR step on the blocks of colour c, one CTA per (block, rhs):
//   alpha_B = <p, r>_B / <p, p>_B (0 if <p, p>_B = 0), x += alpha_B r, r -= alpha_B p
// with p = D_B r.  The block's sums are taken in FP64 across warps (R within a warp).
// Blocks of the other colour keep x and r (there r = p = 0, so alpha_B would be 0).
constexpr int SAP_T = 256;
template <typename R>
__global__ void __launch_bounds__(SAP_T) k_sap_block_mr(cplx<R>* __restrict__ x, cplx<R>* __restrict__ r,
                                                        const cplx<R>* __restrict__ p,
                                                        const unsigned char* __restrict__ colour, int c, int V,
                                                        int nc, int bvol, bool fine) {
  const int B = blockIdx.x;
  if (colour[B] != c) return;
  const long long n = (long long)V * nc;
  const long long base = (long long)blockIdx.y * n;
  const int E = bvol * nc;
  R acc[3] = {R(0), R(0), R(0)};  // Re <p, r>, Im <p, r>, <p, p>
  for (int e = threadIdx.x; e < E; e += SAP_T) {
    const long long o = base + block_elem(B, e, bvol, nc, V, fine);
    const cplx<R> pv = p[o], rv = r[o];
    acc[0] += pv.x * rv.x + pv.y * rv.y;
    acc[1] += pv.x * rv.y - pv.y * rv.x;
    acc[2] += pv.x * pv.x + pv.y * pv.y;
  }
  __shared__ double scratch[(SAP_T / 32) * 3], red[3];
  block_sum_mixed<R, 3>(acc, scratch, red);
  const double pp = red[2];
  const cplx<R> a = pp != 0.0 ? cmk((R)(red[0] / pp), (R)(red[1] / pp)) : czero<R>();
  for (int e = threadIdx.x; e < E; e += SAP_T) {
    const long long o = base + block_elem(B, e, bvol, nc, V, fine);
    const cplx<R> rv = r[o];
    cmac(x[o], a, rv);
    r[o] = rv - cmul(a, p[o]);
  }
}
template <typename R>
void launch_sap_block_mr(cplx<R>* x, cplx<R>* r, const cplx<R>* p, const unsigned char* colour, int c, int V, int nc,
                         int bvol, bool fine, int nrhs, cudaStream_t st) {
  k_sap_block_mr<R><<<dim3(V / bvol, nrhs), SAP_T, 0, st>>>(x, r, p, colour, c, V, nc, bvol, fine);
  WCMG_LAUNCH_CHECK();
}

#define WCMG_INST(R)                                                                                            \
  template void launch_sap_residual<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const unsigned char*, int, int, \
                                       int, int, bool, int, cudaStream_t);                                      \
  template void launch_sap_block_mr<R>(cplx<R>*, cplx<R>*, const cplx<R>*, const unsigned char*, int, int, int,  \
                                       int, bool, int, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST

}  // namespace wcmg
