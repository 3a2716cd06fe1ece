// Intergrid transfers (Sec. 2.1 Aggregation) with chirality-split near-null
// vectors (Sec. 2.2), and FP64 block orthonormalisation of those vectors.
//
//   restrict (Sec. 3 blockProject):
//     phi(x_c)[s*Nvec + i] = sum_{x in B(x_c)} sum_{c in chirality s} conj(v_i(x)_c) psi(x)_c
//   prolong:
//     psi(x)_c = sum_i v_i(x)_c phi(x_c(x))[s(c)*Nvec + i]
// The chiral halves of v_i are stored once (not doubled with zeros as in the
// paper's Grid version, Sec. 2.2): the projection is the component range.
//
// Sites are stored aggregate-major, so aggregate j owns storage sites
// [j |B|, (j+1) |B|): one CTA owns one aggregate and reduces it with a fixed
// shuffle + shared-memory tree (no atomics, no critical region; this is the
// coarse-site threading with a linear site table that Sec. 3 arrives at).
#include "kernels.h"

namespace wcmg {

// element e of chirality s inside aggregate blk -> offset within a field
__device__ __forceinline__ long long elem_addr(bool fine, int blk, int e, int s, int Vf, int nc, int bvol) {
  const int half = nc >> 1;
  if (fine) {
    const int c = s * half + e / bvol, site = blk * bvol + e % bvol;
    return (long long)c * Vf + site;
  }
  const int site = blk * bvol + e / half, c = s * half + e % half;
  return (long long)site * nc + c;
}

template <typename R, int RR, int NV>
__global__ void __launch_bounds__(256) k_restrict(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                  const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                  int nvec, int nrhs, bool fine) {
  using T = cplx<R>;
  __shared__ T scratch[8 * RR * NV];
  __shared__ T red[RR * NV];
  const int blk = blockIdx.x, r0 = blockIdx.y * RR;
  const int half = nc >> 1, nelem = bvol * half, nb = 2 * nvec;
  const int Vc = Vf / bvol;
  const long long fstride = (long long)Vf * nc;
  for (int s = 0; s < 2; ++s) {
    for (int i0 = 0; i0 < nvec; i0 += NV) {
      T acc[RR * NV];
#pragma unroll
      for (int k = 0; k < RR * NV; ++k) acc[k] = czero<R>();
      for (int e = threadIdx.x; e < nelem; e += blockDim.x) {
        const long long a = elem_addr(fine, blk, e, s, Vf, nc, bvol);
        T p[RR];
#pragma unroll
        for (int r = 0; r < RR; ++r) p[r] = (r0 + r < nrhs) ? in[(r0 + r) * fstride + a] : czero<R>();
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          if (i0 + i < nvec) {
            const T v = vecs[(i0 + i) * fstride + a];
#pragma unroll
            for (int r = 0; r < RR; ++r) cjmac(acc[r * NV + i], v, p[r]);
          }
        }
      }
      block_sum_many<T>(acc, RR * NV, scratch, red);
      for (int k = threadIdx.x; k < RR * NV; k += blockDim.x) {
        const int r = k / NV, i = k % NV;
        if (r0 + r < nrhs && i0 + i < nvec)
          out[((long long)(r0 + r) * Vc + blk) * nb + s * nvec + i0 + i] = red[k];
      }
      __syncthreads();
    }
  }
}

template <typename R, int RR>
__global__ void __launch_bounds__(256) k_prolong(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ cin,
                                                 const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                 int nvec, int nrhs, bool fine) {
  using T = cplx<R>;
  extern __shared__ unsigned char smem_raw[];
  T* phi = reinterpret_cast<T*>(smem_raw);  // [RR][nb]
  const int blk = blockIdx.x, r0 = blockIdx.y * RR;
  const int nb = 2 * nvec, half = nc >> 1, Vc = Vf / bvol;
  const long long fstride = (long long)Vf * nc;
  for (int k = threadIdx.x; k < RR * nb; k += blockDim.x) {
    const int r = k / nb, c = k % nb;
    phi[k] = (r0 + r < nrhs) ? cin[((long long)(r0 + r) * Vc + blk) * nb + c] : czero<R>();
  }
  __syncthreads();
  const int nelem = bvol * nc;
  for (int e = threadIdx.x; e < nelem; e += blockDim.x) {
    long long a;
    int c;
    if (fine) { c = e / bvol; a = (long long)c * Vf + blk * bvol + e % bvol; }
    else { c = e % nc; a = (long long)(blk * bvol + e / nc) * nc + c; }
    const int s = c / half;
    T acc[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) acc[r] = czero<R>();
    for (int i = 0; i < nvec; ++i) {
      const T v = vecs[i * fstride + a];
#pragma unroll
      for (int r = 0; r < RR; ++r) cmac(acc[r], v, phi[r * nb + s * nvec + i]);
    }
#pragma unroll
    for (int r = 0; r < RR; ++r)
      if (r0 + r < nrhs) out[(r0 + r) * fstride + a] = acc[r];
  }
}

template <typename R>
void launch_restrict(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                     int nrhs, bool fine, cudaStream_t st) {
  const int Vc = Vf / bvol;
  if (nrhs >= 4) {
    k_restrict<R, 4, 4><<<dim3(Vc, (nrhs + 3) / 4), 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine);
  } else {
    k_restrict<R, 1, 8><<<dim3(Vc, nrhs), 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine);
  }
  WCMG_LAUNCH_CHECK();
}

template <typename R>
void launch_prolong(cplx<R>* out, const cplx<R>* coarse, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                    int nrhs, bool fine, cudaStream_t st) {
  const int Vc = Vf / bvol, nb = 2 * nvec;
  if (nrhs >= 4) {
    k_prolong<R, 4><<<dim3(Vc, (nrhs + 3) / 4), 256, 4 * nb * sizeof(cplx<R>), st>>>(out, coarse, vecs, Vf, nc, bvol,
                                                                                   nvec, nrhs, fine);
  } else {
    k_prolong<R, 1><<<dim3(Vc, nrhs), 256, nb * sizeof(cplx<R>), st>>>(out, coarse, vecs, Vf, nc, bvol, nvec, nrhs,
                                                                         fine);
  }
  WCMG_LAUNCH_CHECK();
}

// ---------------- block orthonormalisation (K6, FP64) ----------------
// One CTA per (aggregate, chirality).  Column k of the panel is orthogonalised
// against columns 0..k-1 by classical Gram-Schmidt applied twice (CGS2), then
// normalised; in exact arithmetic this is the Q factor with positive real
// diag(R).  Each thread keeps its panel elements of column k in registers.
constexpr int ORTHO_MAXV = 32;
constexpr int ORTHO_MAXE = 8;

__global__ void __launch_bounds__(256) k_block_ortho(double2* __restrict__ vecs, int Vf, int nc, int bvol, int nvec,
                                                     bool fine, int* __restrict__ err) {
  __shared__ double2 scratch[8 * ORTHO_MAXV];
  __shared__ double2 red[ORTHO_MAXV];
  __shared__ double dscratch[8];
  __shared__ double dred[1];
  const int blk = blockIdx.x, s = blockIdx.y;
  const int nelem = bvol * (nc >> 1);
  const long long fstride = (long long)Vf * nc;
  long long addr[ORTHO_MAXE];
#pragma unroll
  for (int q = 0; q < ORTHO_MAXE; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    addr[q] = e < nelem ? elem_addr(fine, blk, e, s, Vf, nc, bvol) : -1;
  }
  for (int k = 0; k < nvec; ++k) {
    double2 a[ORTHO_MAXE];
#pragma unroll
    for (int q = 0; q < ORTHO_MAXE; ++q) a[q] = addr[q] >= 0 ? vecs[k * fstride + addr[q]] : make_double2(0, 0);
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      double2 part[ORTHO_MAXV];
#pragma unroll
      for (int i = 0; i < ORTHO_MAXV; ++i) part[i] = make_double2(0, 0);
#pragma unroll
      for (int i = 0; i < ORTHO_MAXV; ++i) {
        if (i < k) {
#pragma unroll
          for (int q = 0; q < ORTHO_MAXE; ++q)
            if (addr[q] >= 0) cjmac(part[i], vecs[i * fstride + addr[q]], a[q]);
        }
      }
      block_sum_many<double2>(part, k, scratch, red);
#pragma unroll
      for (int i = 0; i < ORTHO_MAXV; ++i) {
        if (i < k) {
          const double2 r = red[i];
#pragma unroll
          for (int q = 0; q < ORTHO_MAXE; ++q)
            if (addr[q] >= 0) a[q] -= cmul(r, vecs[i * fstride + addr[q]]);
        }
      }
      __syncthreads();
    }
    double n2 = 0;
#pragma unroll
    for (int q = 0; q < ORTHO_MAXE; ++q) n2 += cnorm2(a[q]);
    block_sum_many<double>(&n2, 1, dscratch, dred);
    const double nrm = sqrt(dred[0]);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (threadIdx.x == 0) *err = 1;
    }
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
#pragma unroll
    for (int q = 0; q < ORTHO_MAXE; ++q)
      if (addr[q] >= 0) vecs[k * fstride + addr[q]] = inv * a[q];
    __syncthreads();
  }
}

void launch_block_ortho(double2* vecs, int Vf, int nc, int bvol, int nvec, bool fine, int* err, cudaStream_t st) {
  const int nelem = bvol * (nc / 2);
  if (nvec > ORTHO_MAXV) throw Error(-1, "block orthonormalisation supports nvec <= 32");
  if (nelem > 256 * ORTHO_MAXE) throw Error(-1, "aggregate too large for block orthonormalisation");
  k_block_ortho<<<dim3(Vf / bvol, 2), 256, 0, st>>>(vecs, Vf, nc, bvol, nvec, fine, err);
  WCMG_LAUNCH_CHECK();
}

// ---------------- chirality-split columns of P ----------------
template <typename R>
__global__ void k_make_columns(cplx<R>* __restrict__ cols, const cplx<R>* __restrict__ vecs, int Vf, int nc,
                               int nvec, int b0, bool fine) {
  const long long fsize = (long long)Vf * nc;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (e >= fsize) return;
  const int b = b0 + j, s = b / nvec, i = b % nvec;
  const int c = fine ? (int)(e / Vf) : (int)(e % nc);
  const bool keep = (c / (nc >> 1)) == s;
  cols[j * fsize + e] = keep ? vecs[i * fsize + e] : czero<R>();
}

template <typename R>
void launch_make_columns(cplx<R>* cols, const cplx<R>* vecs, int Vf, int nc, int nvec, int b0, int ncols, bool fine,
                         cudaStream_t st) {
  const long long fsize = (long long)Vf * nc;
  k_make_columns<R><<<dim3(nblk(fsize, 256), ncols), 256, 0, st>>>(cols, vecs, Vf, nc, nvec, b0, fine);
  WCMG_LAUNCH_CHECK();
}

#define WCMG_INST(R)                                                                                            \
  template void launch_restrict<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, int, int, int, int, int, bool,     \
                                   cudaStream_t);                                                               \
  template void launch_prolong<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, int, int, int, int, int, bool,      \
                                  cudaStream_t);                                                                \
  template void launch_make_columns<R>(cplx<R>*, const cplx<R>*, int, int, int, int, int, bool, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST

}  // namespace wcmg
