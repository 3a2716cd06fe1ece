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
#include "dfloat.cuh"

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

// Face restriction (coarsening): only the sites of an aggregate whose neighbour
// across face `fd` (2 mu for +mu, 2 mu + 1 for -mu) lies in the next aggregate.
struct FaceSel {
  int fd;     // -1: whole aggregate
  int b[4];   // aggregate extents
};

// local site of the aggregate for index f over the selected sites
__device__ __forceinline__ int face_site(const FaceSel& fs, int f) {
  if (fs.fd < 0) return f;
  const int mu = fs.fd >> 1, fixed = (fs.fd & 1) ? 0 : fs.b[mu] - 1;
  int l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k == mu) { l[k] = fixed; continue; }
    l[k] = f % fs.b[k];
    f /= fs.b[k];
  }
  return l[0] + fs.b[0] * (l[1] + fs.b[1] * (l[2] + fs.b[2] * l[3]));
}

// One CTA (8 warps) per (aggregate, tile of RR right-hand sides).  The CTA walks
// the selected elements of one chirality in chunks of 256; each chunk of the RR
// fine fields is staged once in shared memory.  Warp w owns the near-null
// vectors i = w, w + 8, ... (VPW of them): every vector element is loaded once
// from global memory and each lane keeps RR x VPW complex partial sums; the only
// reduction is a warp shuffle at the end.
template <typename R, int RR, int VPW>
__global__ void __launch_bounds__(256) k_restrict(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                  const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                  int nvec, int nrhs, bool fine, FaceSel fs) {
  using T = cplx<R>;
  constexpr int CH = 256;
  __shared__ T ps[RR][CH];
  __shared__ int off_s[CH];
  // rhs tile fastest in the grid: CTAs running together share an aggregate's vectors in L2
  const int ntile = (nrhs + RR - 1) / RR;
  const int blk = blockIdx.x / ntile, r0 = (blockIdx.x % ntile) * RR, s = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int half = nc >> 1, nb = 2 * nvec;
  const int nsite = fs.fd < 0 ? bvol : bvol / fs.b[fs.fd >> 1];
  const int nelem = nsite * half;
  const int Vc = Vf / bvol;
  const long long fstride = (long long)Vf * nc;
  const T* vb[VPW];
#pragma unroll
  for (int j = 0; j < VPW; ++j) {
    const int i = warp + nw * j;
    vb[j] = i < nvec ? vecs + i * fstride : nullptr;
  }
  T acc[RR][VPW];
#pragma unroll
  for (int r = 0; r < RR; ++r)
#pragma unroll
    for (int j = 0; j < VPW; ++j) acc[r][j] = czero<R>();
  for (int c0 = 0; c0 < nelem; c0 += CH) {
    // stage: element -> offset (fast index of the layout first), and the rhs values
    const int e = c0 + threadIdx.x;
    if (e < nelem) {
      int c, f;
      if (fine) { c = s * half + e / nsite; f = e % nsite; }
      else { f = e / half; c = s * half + e % half; }
      const int site = blk * bvol + face_site(fs, f);
      const int a = fine ? c * Vf + site : site * nc + c;
      off_s[threadIdx.x] = a;
#pragma unroll
      for (int r = 0; r < RR; ++r) ps[r][threadIdx.x] = (r0 + r < nrhs) ? in[(r0 + r) * fstride + a] : czero<R>();
    }
    __syncthreads();
    const int cn = min(CH, nelem - c0);
#pragma unroll 4
    for (int t = lane; t < cn; t += 32) {
      const int a = off_s[t];
#pragma unroll
      for (int j = 0; j < VPW; ++j) {
        if (vb[j]) {
          const T v = vb[j][a];
#pragma unroll
          for (int r = 0; r < RR; ++r) cjmac(acc[r][j], v, ps[r][t]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < RR; ++r)
#pragma unroll
    for (int j = 0; j < VPW; ++j) {
      const T t = warp_sum(acc[r][j]);
      const int i = warp + nw * j;
      if (lane == 0 && i < nvec && r0 + r < nrhs) out[((long long)(r0 + r) * Vc + blk) * nb + s * nvec + i] = t;
    }
}

template <typename R, int RR>
__global__ void __launch_bounds__(256) k_prolong(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ cin,
                                                 const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                 int nvec, int nrhs, bool fine) {
  using T = cplx<R>;
  extern __shared__ unsigned char smem_raw[];
  T* phi = reinterpret_cast<T*>(smem_raw);  // [RR][nb]
  const int ntile = (nrhs + RR - 1) / RR;  // rhs tile fastest: the vectors are shared in L2
  const int blk = blockIdx.x / ntile, r0 = (blockIdx.x % ntile) * RR;
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

// Few right-hand sides: one warp per (aggregate, chirality, vector) dot
// product.  A CTA holds 8 warps = 8 vectors of one (aggregate, chirality), so
// the fine-field entries they all read come from L1; each lane streams its
// elements of one vector with UNR independent loads in flight.  No shared
// memory, no block barrier, a warp shuffle at the end.  Fine layout: the
// aggregate's chirality half is `half` runs of bvol consecutive sites.
template <typename R, int UNR>
__global__ void __launch_bounds__(256) k_restrict_few(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                      const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                      int nvec, int nrhs, bool fine, FaceSel fs) {
  using T = cplx<R>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int vgroups = (nvec + 7) / 8;
  const int g = blockIdx.x % vgroups;
  const int s = (blockIdx.x / vgroups) & 1;
  const int blk = blockIdx.x / (2 * vgroups);
  const int i = g * 8 + warp;
  if (i >= nvec) return;
  const int half = nc >> 1, nb = 2 * nvec;
  const int Vc = Vf / bvol;
  const long long fstride = (long long)Vf * nc;
  const T* v = vecs + i * fstride;
  const bool plain = fine && fs.fd < 0;
  const int nsite = fs.fd < 0 ? bvol : bvol / fs.b[fs.fd >> 1];
  const int nelem = nsite * half;
  for (int r = 0; r < nrhs; ++r) {
    const T* p = in + r * fstride;
    T acc = czero<R>();
    if (plain) {
      // element (c, site): offset (s half + c) Vf + blk bvol + site
      const long long base = (long long)(s * half) * Vf + (long long)blk * bvol;
      for (int c = 0; c < half; ++c) {
        const long long rowb = base + (long long)c * Vf;
        for (int q0 = lane; q0 < bvol; q0 += 32 * UNR) {
          T vv[UNR], pp[UNR];
#pragma unroll
          for (int u = 0; u < UNR; ++u) {
            const int q = q0 + 32 * u;
            vv[u] = q < bvol ? v[rowb + q] : czero<R>();
            pp[u] = q < bvol ? p[rowb + q] : czero<R>();
          }
#pragma unroll
          for (int u = 0; u < UNR; ++u) cjmac(acc, vv[u], pp[u]);
        }
      }
    } else {
      for (int e0 = lane; e0 < nelem; e0 += 32 * UNR) {
        T vv[UNR], pp[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int e = e0 + 32 * u;
          vv[u] = czero<R>();
          pp[u] = czero<R>();
          if (e < nelem) {
            int c, f;
            if (fine) { c = s * half + e / nsite; f = e % nsite; }
            else { f = e / half; c = s * half + e % half; }
            const int site = blk * bvol + face_site(fs, f);
            const long long a = fine ? (long long)c * Vf + site : (long long)site * nc + c;
            vv[u] = v[a];
            pp[u] = p[a];
          }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) cjmac(acc, vv[u], pp[u]);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) out[((long long)r * Vc + blk) * nb + s * nvec + i] = acc;
  }
}

template <typename R>
static void restrict_few(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                         int nrhs, bool fine, const FaceSel& fs, cudaStream_t st) {
  const int vgroups = (nvec + 7) / 8;
  const unsigned grid = (unsigned)((Vf / bvol) * 2 * vgroups);
  k_restrict_few<R, 8><<<grid, 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  WCMG_LAUNCH_CHECK();
}

// Many right-hand sides (the coarsening's column fields, the setup batches): a
// register-blocked GEMM per (aggregate, chirality): out[(s, i)][r] =
// sum_e conj(v_i[e]) in_r[e] over the aggregate's (selected) elements e of
// chirality s.  Each K-chunk of RST_KT elements of all vectors and all rhs of the
// tile is staged once in shared memory; thread (ti, tr) of the 8 x TR threads owns
// vectors ti + 8 q (q < VI) and rhs tr + TR p (p < RT): VI x RT complex accumulators
// per thread, VI + RT shared loads per element for VI x RT complex MACs.
// Staging: thread t loads element t % RST_KT of the chunk (coalesced along the
// aggregate's sites) for rows t / RST_KT + ROWS j; the next chunk is loaded into
// registers while the current one is multiplied.  Shared rows are padded to an odd
// number of complex entries, so the staging stores (one row entry per lane) hit
// distinct banks.
constexpr int RST_KT = 32;
template <typename R, int VI, int RT, int TR>
__global__ void __launch_bounds__(8 * TR) k_restrict_gemm(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                          const cplx<R>* __restrict__ vecs, int Vf, int nc, int bvol,
                                                          int nvec, int nrhs, bool fine, FaceSel fs) {
  using T = cplx<R>;
  constexpr int NTH = 8 * TR;
  constexpr int NT = TR * RT;  // rhs per CTA
  constexpr int NV = 8 * VI;   // vectors per CTA
  constexpr int ROWS = NTH / RST_KT;
  static_assert(NTH % RST_KT == 0, "staging rows");
  constexpr int XJ = (NV + ROWS - 1) / ROWS, TJ = (NT + ROWS - 1) / ROWS;
  constexpr int XP = NV | 1, TP = NT | 1;  // odd row strides
  __shared__ T Xs[RST_KT][XP];
  __shared__ T Ts[RST_KT][TP];
  const int blk = blockIdx.x, s = blockIdx.y, r0 = blockIdx.z * NT;
  const int tid = threadIdx.x, ti = tid / TR, tr = tid % TR;
  const int kown = tid % RST_KT, row0 = tid / RST_KT;
  const int half = nc >> 1, nb = 2 * nvec;
  const int nsite = fs.fd < 0 ? bvol : bvol / fs.b[fs.fd >> 1];
  const int nelem = nsite * half;
  const int Vc = Vf / bvol;
  const long long fstride = (long long)Vf * nc;
  T xr[XJ], trr[TJ];
  auto fetch = [&](int c0) {
    const int e = c0 + kown;
    long long a = -1;
    if (e < nelem) {
      int c, f;
      if (fine) { c = s * half + e / nsite; f = e % nsite; }
      else { f = e / half; c = s * half + e % half; }
      const int site = blk * bvol + face_site(fs, f);
      a = fine ? (long long)c * Vf + site : (long long)site * nc + c;
    }
#pragma unroll
    for (int j = 0; j < XJ; ++j) {
      const int i = row0 + ROWS * j;
      xr[j] = (a >= 0 && i < nvec) ? vecs[i * fstride + a] : czero<R>();
    }
#pragma unroll
    for (int j = 0; j < TJ; ++j) {
      const int r = row0 + ROWS * j;
      trr[j] = (a >= 0 && r < NT && r0 + r < nrhs) ? in[(r0 + r) * fstride + a] : czero<R>();
    }
  };
  T acc[VI][RT];
#pragma unroll
  for (int q = 0; q < VI; ++q)
#pragma unroll
    for (int p = 0; p < RT; ++p) acc[q][p] = czero<R>();
  fetch(0);
  for (int c0 = 0; c0 < nelem; c0 += RST_KT) {
#pragma unroll
    for (int j = 0; j < XJ; ++j)
      if (row0 + ROWS * j < NV) Xs[kown][row0 + ROWS * j] = xr[j];
#pragma unroll
    for (int j = 0; j < TJ; ++j)
      if (row0 + ROWS * j < NT) Ts[kown][row0 + ROWS * j] = trr[j];
    __syncthreads();
    if (c0 + RST_KT < nelem) fetch(c0 + RST_KT);
#pragma unroll 4
    for (int kk = 0; kk < RST_KT; ++kk) {
      T x[VI], t[RT];
#pragma unroll
      for (int q = 0; q < VI; ++q) x[q] = Xs[kk][ti + 8 * q];
#pragma unroll
      for (int p = 0; p < RT; ++p) t[p] = Ts[kk][tr + TR * p];
#pragma unroll
      for (int q = 0; q < VI; ++q)
#pragma unroll
        for (int p = 0; p < RT; ++p) cjmac(acc[q][p], x[q], t[p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < VI; ++q)
#pragma unroll
    for (int p = 0; p < RT; ++p) {
      const int i = ti + 8 * q, r = r0 + tr + TR * p;
      if (i < nvec && r < nrhs) out[((long long)r * Vc + blk) * nb + s * nvec + i] = acc[q][p];
    }
}

template <typename R, int VI, int RT>
static void restrict_gemm_v(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol,
                            int nvec, int nrhs, bool fine, const FaceSel& fs, cudaStream_t st) {
  constexpr int TR = 16;
  const dim3 grid(Vf / bvol, 2, (nrhs + TR * RT - 1) / (TR * RT));
  k_restrict_gemm<R, VI, RT, TR><<<grid, 8 * TR, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  WCMG_LAUNCH_CHECK();
}

template <typename R, int VI>
static void restrict_gemm_vi(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol,
                             int nvec, int nrhs, bool fine, const FaceSel& fs, cudaStream_t st) {
  // rhs per CTA 16 x RT: 32 (<= 32 rhs), 48 (more; the 48 column fields of nbasis 48)
  if (nrhs <= 32) restrict_gemm_v<R, VI, 2>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else restrict_gemm_v<R, VI, 3>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
}

template <typename R>
static void restrict_gemm(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                          int nrhs, bool fine, const FaceSel& fs, cudaStream_t st) {
  const int vi = (nvec + 7) / 8;
  if (vi <= 2) restrict_gemm_vi<R, 2>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else if (vi == 3) restrict_gemm_vi<R, 3>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else restrict_gemm_vi<R, 4>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
}

template <typename R, int RR>
static void restrict_rr(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                        int nrhs, bool fine, const FaceSel& fs, cudaStream_t st) {
  const dim3 grid((Vf / bvol) * ((nrhs + RR - 1) / RR), 2);
  const int vpw = (nvec + 7) / 8;
  if (vpw == 1) k_restrict<R, RR, 1><<<grid, 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  else if (vpw == 2) k_restrict<R, RR, 2><<<grid, 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  else if (vpw == 3) k_restrict<R, RR, 3><<<grid, 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  else k_restrict<R, RR, 4><<<grid, 256, 0, st>>>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
void launch_restrict(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                     int nrhs, bool fine, cudaStream_t st, int face, const int* block) {
  if (nvec > 32) throw Error(-1, "restrict supports nvec <= 32");
  FaceSel fs;
  fs.fd = face;
  for (int k = 0; k < 4; ++k) fs.b[k] = block ? block[k] : 1;
  if (face >= 0 && !block) throw Error(-1, "face restriction needs the aggregate extents");
  if (nrhs >= 16) restrict_gemm<R>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else if (sizeof(R) == 4 && nrhs >= 8) restrict_rr<R, 8>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else if (nrhs >= 4) restrict_rr<R, 4>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
  else restrict_few<R>(coarse, in, vecs, Vf, nc, bvol, nvec, nrhs, fine, fs, st);
}

template <typename R>
void launch_prolong(cplx<R>* out, const cplx<R>* coarse, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                    int nrhs, bool fine, cudaStream_t st) {
  const int Vc = Vf / bvol, nb = 2 * nvec;
  if (nrhs >= 4) {
    k_prolong<R, 4><<<dim3(Vc * ((nrhs + 3) / 4)), 256, 4 * nb * sizeof(cplx<R>), st>>>(out, coarse, vecs, Vf, nc,
                                                                                       bvol, nvec, nrhs, fine);
  } else {
    k_prolong<R, 1><<<dim3(Vc * nrhs), 256, nb * sizeof(cplx<R>), st>>>(out, coarse, vecs, Vf, nc, bvol, nvec,
                                                                           nrhs, fine);
  }
  WCMG_LAUNCH_CHECK();
}

// ---------------- block orthonormalisation (K6, FP64) ----------------
// One CTA per (aggregate, chirality).  Column k of the panel is orthogonalised
// against columns 0..k-1 by classical Gram-Schmidt; one pass leaves inner
// products with the earlier columns of order eps ||a|| / ||a'|| (a' the column
// after the pass), so a second pass is taken only when the first one cancelled
// more than 99 % of the norm (||a'|| < 0.01 ||a||): the result is orthonormal to
// about 100 eps = 2e-14 in FP64 (the selective reorthogonalisation of
// Daniel-Gragg-Kaufman-Stewart with a 0.01 threshold); then it is normalised.  In exact arithmetic this is the Q
// factor with positive real diag(R).  Each thread keeps its MAXE panel elements
// of column k in registers; the previous columns are re-read from L1/L2.
// The loops over earlier columns have run-time trip counts (no predicated-off
// FP64 work); each coefficient is reduced by warp shuffles into shared memory.
template <int MAXE>
__global__ void __launch_bounds__(256, 2) k_block_ortho(double2* __restrict__ vecs, int Vf, int nc, int bvol, int nvec,
                                                     bool fine, int* __restrict__ err) {
  constexpr int MV = 33;  // nvec <= 32, slot 32: squared norm
  __shared__ double2 scratch[8][MV];
  __shared__ double2 red[MV];
  const int blk = blockIdx.x, s = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nelem = bvol * (nc >> 1);
  const long long fstride = (long long)Vf * nc;
  long long addr[MAXE];
#pragma unroll
  for (int q = 0; q < MAXE; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    addr[q] = e < nelem ? elem_addr(fine, blk, e, s, Vf, nc, bvol) : -1;
  }
  // block-wide sums of slots [0, n) and the norm slot
  auto reduce = [&](int n, bool with_norm) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double2 t = scratch[0][i];
      for (int w = 1; w < nw; ++w) t += scratch[w][i];
      red[i] = t;
    }
    if (with_norm && threadIdx.x == 0) {
      double2 t = scratch[0][MV - 1];
      for (int w = 1; w < nw; ++w) t += scratch[w][MV - 1];
      red[MV - 1] = t;
    }
    __syncthreads();
  };
  for (int k = 0; k < nvec; ++k) {
    double2 a[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) a[q] = addr[q] >= 0 ? vecs[k * fstride + addr[q]] : make_double2(0, 0);
    double before2 = 0.0, after2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      // projections <q_i, a> for i < k, eight at a time (one transposing warp reduction)
      for (int i0 = 0; i0 < k; i0 += 8) {
        double2 p[8];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          p[g] = make_double2(0, 0);
          if (i0 + g < k) {
            const double2* qi = vecs + (i0 + g) * fstride;
#pragma unroll
            for (int q = 0; q < MAXE; ++q)
              if (addr[q] >= 0) cjmac(p[g], qi[addr[q]], a[q]);
          }
        }
        warp_sum8_transposed(p, lane);
        const int g = warp_sum8_index(lane);
        if ((lane & 3) == 0 && i0 + g < k) scratch[warp][i0 + g] = p[0];
      }
      double n0 = 0;
#pragma unroll
      for (int q = 0; q < MAXE; ++q) n0 += cnorm2(a[q]);
      n0 = warp_sum(n0);
      if (lane == 0) scratch[warp][MV - 1] = make_double2(n0, 0);
      reduce(k, true);
      if (pass == 0) before2 = red[MV - 1].x;
      for (int i = 0; i < k; ++i) {
        const double2 r = red[i];
        const double2* qi = vecs + i * fstride;
#pragma unroll
        for (int q = 0; q < MAXE; ++q)
          if (addr[q] >= 0) cnmac(a[q], r, qi[addr[q]]);
      }
      double n2 = 0;
#pragma unroll
      for (int q = 0; q < MAXE; ++q) n2 += cnorm2(a[q]);
      n2 = warp_sum(n2);
      if (lane == 0) scratch[warp][MV - 1] = make_double2(n2, 0);
      reduce(0, true);
      after2 = red[MV - 1].x;
      if (k == 0 || after2 >= 1e-4 * before2) break;  // uniform over the block
    }
    const double nrm = sqrt(after2);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (threadIdx.x == 0) *err = 1;
    }
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
#pragma unroll
    for (int q = 0; q < MAXE; ++q)
      if (addr[q] >= 0) vecs[k * fstride + addr[q]] = inv * a[q];
    __syncthreads();
  }
}

// ---------------- block orthonormalisation in double-float arithmetic ----------------
// The same Gram-Schmidt (classical, with the selective second pass and the
// normalisation of k_block_ortho) with every multiply-add on the FP32 pipe in
// double-float ("DF") form: a value is the unevaluated sum h + l of two floats
// (|l| <= ulp(h) / 2 once normalised: 48 significand bits).  Error-free
// transformations give the exact rounding error of a float sum (Knuth's TwoSum) and
// of a float product (by FMA); the dot products accumulate them as in the
// compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005), so each projection is as accurate as one formed in
// twice the float precision.  The input and the returned Q stay FP64 (the value of
// h + l rounded to double); the Q columns are also kept in DF in `qdf` (float4 per
// complex entry: re.h, re.l, im.h, im.l), from which later columns re-read them.
// FP32 arithmetic runs 64x faster than FP64 on this part, and one DF multiply-add
// costs 12 FP32 operations.


// Input column entry in double-float: from the FP64 field, or, when in32 is given,
// from an FP32 field (exact: the FP32 value with a zero low part, the same as splitting
// that value widened to FP64).
__device__ __forceinline__ dfc ortho_df_input(const double2* vecs, const float2* in32, long long i) {
  if (in32) {
    const float2 v = in32[i];
    return {{v.x, 0.f}, {v.y, 0.f}};
  }
  const double2 v = vecs[i];
  return {df_split(v.x), df_split(v.y)};
}
// Output entry q_k: FP64 (vecs), double-float (qdf, read back by the later columns), and,
// when out32 is given, its FP32 rounding (the FP64 value converted, as a separate
// conversion pass would)
__device__ __forceinline__ void ortho_df_output(double2* vecs, float4* qdf, float2* out32, long long i, dfr re,
                                                dfr im) {
  const double2 v = make_double2(df_to_fast(re), df_to_fast(im));
  vecs[i] = v;
  qdf[i] = make_float4(re.h, re.l, im.h, im.l);
  if (out32) out32[i] = make_float2((float)v.x, (float)v.y);
}

template <int MAXE, int NT, int MINB, int GS>
__global__ void __launch_bounds__(NT, MINB) k_block_ortho_df(double2* __restrict__ vecs, float4* __restrict__ qdf,
                                                             int Vf, int nc, int bvol, int nvec, bool fine,
                                                             int* __restrict__ err, const float2* __restrict__ in32,
                                                             float2* __restrict__ out32) {
  constexpr int MV = 33;  // nvec <= 32, slot 32: squared norm
  __shared__ dfc scratch[NT / 32][MV];
  __shared__ dfc red[MV];
  const int blk = blockIdx.x, s = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nelem = bvol * (nc >> 1);
  const long long fstride = (long long)Vf * nc;
  int addr[MAXE];  // offsets within one field (< 2^31: checked by the launcher)
#pragma unroll
  for (int q = 0; q < MAXE; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    addr[q] = e < nelem ? (int)elem_addr(fine, blk, e, s, Vf, nc, bvol) : -1;
  }
  const dfc zero = {{0.f, 0.f}, {0.f, 0.f}};
  // block-wide DF sums of slots [0, n) and the norm slot
  auto reduce = [&](int n, bool with_norm) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      dfc t = scratch[0][i];
      for (int w = 1; w < nw; ++w) t = dfc_add(t, scratch[w][i]);
      red[i] = t;
    }
    if (with_norm && threadIdx.x == 0) {
      dfc t = scratch[0][MV - 1];
      for (int w = 1; w < nw; ++w) t = dfc_add(t, scratch[w][MV - 1]);
      red[MV - 1] = t;
    }
    __syncthreads();
  };
  auto norm2 = [&](const dfc (&a)[MAXE]) {
    dfr n = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      df_mac(n, a[q].re, a[q].re);
      df_mac(n, a[q].im, a[q].im);
    }
    n = df_warp_sum(df_norm(n));
    if (lane == 0) scratch[warp][MV - 1] = {n, {0.f, 0.f}};
  };
  for (int k = 0; k < nvec; ++k) {
    dfc a[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      if (addr[q] >= 0) {
        a[q] = ortho_df_input(vecs, in32, k * fstride + addr[q]);
      } else {
        a[q] = zero;
      }
    }
    double before2 = 0.0, after2 = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      // projections <q_i, a> for i < k, GS at a time (one transposing warp reduction)
      for (int i0 = 0; i0 < k; i0 += GS) {
        dfc p[GS];
#pragma unroll
        for (int g = 0; g < GS; ++g) {
          p[g] = zero;
          if (i0 + g < k) {
            const float4* qi = qdf + (i0 + g) * fstride;
#pragma unroll
            for (int q = 0; q < MAXE; ++q)
              if (addr[q] >= 0) dfc_cjmac(p[g], dfc_load(qi + addr[q]), a[q]);
          }
          p[g] = dfc_norm(p[g]);
        }
        dfc_warp_sum_transposed<GS>(p, lane);
        const int g = dfc_sum_index<GS>(lane);
        if ((lane & (32 / GS - 1)) == 0 && i0 + g < k) scratch[warp][i0 + g] = p[0];
      }
      norm2(a);
      reduce(k, true);
      if (pass == 0) before2 = df_to_fast(red[MV - 1].re);
      for (int i = 0; i < k; ++i) {
        const dfc r = red[i];
        const float4* qi = qdf + i * fstride;
#pragma unroll
        for (int q = 0; q < MAXE; ++q)
          if (addr[q] >= 0) dfc_nmac(a[q], r, dfc_load(qi + addr[q]));
      }
#pragma unroll
      for (int q = 0; q < MAXE; ++q) a[q] = dfc_norm(a[q]);
      norm2(a);
      reduce(0, true);
      after2 = df_to_fast(red[MV - 1].re);
      if (k == 0 || after2 >= 1e-4 * before2) break;  // uniform over the block
    }
    const double nrm = sqrt(after2);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (threadIdx.x == 0) *err = 1;
    }
    const dfr inv = df_split(nrm > 0.0 ? 1.0 / nrm : 0.0);
#pragma unroll
    for (int q = 0; q < MAXE; ++q)
      if (addr[q] >= 0) {
        const dfr re = df_mul(a[q].re, inv), im = df_mul(a[q].im, inv);
        ortho_df_output(vecs, qdf, out32, k * fstride + addr[q], re, im);
      }
    __syncthreads();
  }
}


// Columns in pairs: the first Gram-Schmidt pass of columns k and k + 1 against the
// finished columns Q_{<k} is one sweep over Q_{<k} (each re-read of Q serves both
// columns), which halves the kernel's dominant traffic, the re-reads of earlier Q
// columns.  Column k then follows the single-column kernel (selective second pass,
// normalisation); column k + 1 is projected on the new q_k from registers, and its
// selective second pass (against all of Q_{<=k}) is taken when the whole projection
// cancelled more than 99 % of its norm, the same test as before.  The Q factor is the
// same up to rounding; the second passes are rare for near-null candidates.
template <int MAXE, int NT, int MINB, int GS>
__global__ void __launch_bounds__(NT, MINB) k_block_ortho_df2(double2* __restrict__ vecs, float4* __restrict__ qdf,
                                                              int Vf, int nc, int bvol, int nvec, bool fine,
                                                              int* __restrict__ err, const float2* __restrict__ in32,
                                                              float2* __restrict__ out32) {
  constexpr int MV = 33;  // nvec <= 32, slot 32: squared norm
  __shared__ dfc scratch[2][NT / 32][MV];
  __shared__ dfc red[2][MV];
  const int blk = blockIdx.x, s = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nelem = bvol * (nc >> 1);
  const long long fstride = (long long)Vf * nc;
  int addr[MAXE];
#pragma unroll
  for (int q = 0; q < MAXE; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    addr[q] = e < nelem ? (int)elem_addr(fine, blk, e, s, Vf, nc, bvol) : -1;
  }
  const dfc zero = {{0.f, 0.f}, {0.f, 0.f}};
  // block-wide DF sums of the slots [0, n) of columns [0, ncol) and of their norm slots
  auto reduce = [&](int n, int ncol) {
    __syncthreads();
    for (int i = threadIdx.x; i < ncol * MV; i += blockDim.x) {
      const int c = i / MV, j = i - c * MV;
      if (j < n || j == MV - 1) {
        dfc t = scratch[c][0][j];
        for (int w = 1; w < nw; ++w) t = dfc_add(t, scratch[c][w][j]);
        red[c][j] = t;
      }
    }
    __syncthreads();
  };
  auto norm2 = [&](const dfc (&a)[MAXE], int c) {
    dfr n = {0.f, 0.f};
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      df_mac(n, a[q].re, a[q].re);
      df_mac(n, a[q].im, a[q].im);
    }
    n = df_warp_sum(df_norm(n));
    if (lane == 0) scratch[c][warp][MV - 1] = {n, {0.f, 0.f}};
  };
  // projections of columns a0 (and a1 when two) on Q_{<k} into scratch[0 / 1][.][0, k)
  auto project = [&](const dfc (&a0)[MAXE], const dfc (&a1)[MAXE], int k, bool two) {
    for (int i0 = 0; i0 < k; i0 += GS) {
      dfc p0[GS], p1[GS];
#pragma unroll
      for (int g = 0; g < GS; ++g) {
        p0[g] = zero;
        p1[g] = zero;
        if (i0 + g < k) {
          const float4* qi = qdf + (i0 + g) * fstride;
#pragma unroll
          for (int q = 0; q < MAXE; ++q)
            if (addr[q] >= 0) {
              const dfc qv = dfc_load(qi + addr[q]);
              dfc_cjmac(p0[g], qv, a0[q]);
              if (two) dfc_cjmac(p1[g], qv, a1[q]);
            }
        }
        p0[g] = dfc_norm(p0[g]);
        p1[g] = dfc_norm(p1[g]);
      }
      dfc_warp_sum_transposed<GS>(p0, lane);
      const int g = dfc_sum_index<GS>(lane);
      const bool w0 = (lane & (32 / GS - 1)) == 0 && i0 + g < k;
      if (w0) scratch[0][warp][i0 + g] = p0[0];
      if (two) {
        dfc_warp_sum_transposed<GS>(p1, lane);
        if (w0) scratch[1][warp][i0 + g] = p1[0];
      }
    }
  };
  // a0 -= sum_i red[0][i] q_i (and a1 with red[1]) over i < k
  auto subtract = [&](dfc (&a0)[MAXE], dfc (&a1)[MAXE], int k, bool two) {
    for (int i = 0; i < k; ++i) {
      const dfc r0 = red[0][i], r1 = red[1][i];
      const float4* qi = qdf + i * fstride;
#pragma unroll
      for (int q = 0; q < MAXE; ++q)
        if (addr[q] >= 0) {
          const dfc qv = dfc_load(qi + addr[q]);
          dfc_nmac(a0[q], r0, qv);
          if (two) dfc_nmac(a1[q], r1, qv);
        }
    }
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      a0[q] = dfc_norm(a0[q]);
      if (two) a1[q] = dfc_norm(a1[q]);
    }
  };
  auto load_col = [&](dfc (&a)[MAXE], int k) {
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      if (addr[q] >= 0) {
        a[q] = ortho_df_input(vecs, in32, k * fstride + addr[q]);
      } else {
        a[q] = zero;
      }
    }
  };
  // normalise a by the norm whose square is n2 and store it as column k
  auto finish = [&](dfc (&a)[MAXE], double n2, int k) {
    const double nrm = sqrt(n2);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      if (threadIdx.x == 0) *err = 1;
    }
    const dfr inv = df_split(nrm > 0.0 ? 1.0 / nrm : 0.0);
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      const dfr re = df_mul(a[q].re, inv), im = df_mul(a[q].im, inv);
      a[q] = {re, im};
      if (addr[q] >= 0) ortho_df_output(vecs, qdf, out32, k * fstride + addr[q], re, im);
    }
  };
  dfc none[MAXE];
#pragma unroll
  for (int q = 0; q < MAXE; ++q) none[q] = zero;
  for (int k = 0; k < nvec; k += 2) {
    const bool two = k + 1 < nvec;
    dfc a0[MAXE], a1[MAXE];
    load_col(a0, k);
    if (two) load_col(a1, k + 1);
    else
#pragma unroll
      for (int q = 0; q < MAXE; ++q) a1[q] = zero;
    // first pass of both columns against Q_{<k}, norms before
    project(a0, a1, k, two);
    norm2(a0, 0);
    if (two) norm2(a1, 1);
    reduce(k, two ? 2 : 1);
    const double before0 = df_to_fast(red[0][MV - 1].re);
    const double before1 = two ? df_to_fast(red[1][MV - 1].re) : 0.0;
    subtract(a0, a1, k, two);
    norm2(a0, 0);
    reduce(0, 1);
    double after0 = df_to_fast(red[0][MV - 1].re);
    if (k > 0 && after0 < 1e-4 * before0) {  // second pass of column k (uniform)
      project(a0, none, k, false);
      norm2(a0, 0);
      reduce(k, 1);
      subtract(a0, none, k, false);
      norm2(a0, 0);
      reduce(0, 1);
      after0 = df_to_fast(red[0][MV - 1].re);
    }
    finish(a0, after0, k);  // a0 now holds q_k
    if (!two) {
      __syncthreads();
      continue;
    }
    // column k + 1: projection on q_k from registers (summed in slot 0 of column 0)
    {
      dfc p = zero;
#pragma unroll
      for (int q = 0; q < MAXE; ++q)
        if (addr[q] >= 0) dfc_cjmac(p, a0[q], a1[q]);
      p = dfc_norm(p);
      p = {df_warp_sum(p.re), df_warp_sum(p.im)};
      if (lane == 0) scratch[0][warp][0] = p;
      reduce(1, 1);
    }
    {
      const dfc r = red[0][0];
#pragma unroll
      for (int q = 0; q < MAXE; ++q) {
        dfc_nmac(a1[q], r, a0[q]);
        a1[q] = dfc_norm(a1[q]);
      }
    }
    norm2(a1, 1);
    reduce(0, 2);
    double after1 = df_to_fast(red[1][MV - 1].re);
    if (after1 < 1e-4 * before1) {  // second pass of column k + 1 against Q_{<=k} (uniform)
      project(a1, none, k + 1, false);  // q_k is stored: read it back with the others
      norm2(a1, 0);
      reduce(k + 1, 1);
      subtract(a1, none, k + 1, false);
      norm2(a1, 0);
      reduce(0, 1);
      after1 = df_to_fast(red[0][MV - 1].re);
    }
    finish(a1, after1, k + 1);
    __syncthreads();
  }
}


void launch_block_ortho_df(double2* vecs, float4* qdf, int Vf, int nc, int bvol, int nvec, bool fine, int* err,
                           cudaStream_t st, const float2* in32, float2* out32) {
  const int nelem = bvol * (nc / 2);
  if (nvec > 32) throw Error(-1, "block orthonormalisation supports nvec <= 32");
  if (nelem > 256 * 8) throw Error(-1, "aggregate too large for block orthonormalisation");
  if ((long long)Vf * nc >= (1LL << 31)) throw Error(-1, "block orthonormalisation: field too large");
  const dim3 grid(Vf / bvol, 2);
  // Launch shapes measured on 32^3x64 (panels of 1536 x 24; threads x rows per thread,
  // CTAs per SM, columns per warp reduction): one column at a time, 512 x 3, 4 CTAs (64
  // warps, 32 registers), groups of 4: 49 ms per call; the same at 3 CTAs: 53 ms; 3 CTAs,
  // groups of 8: 58 ms; 256 x 6, 3 CTAs: 73 ms; 768 x 2, 2 CTAs: 63 ms; 384 x 4, 3 CTAs:
  // 61 ms.  Columns in pairs, 512 x 3, 2 CTAs (64 registers), groups of 2: 47 ms (16^3x32:
  // 3.5 against 3.8 ms).  The kernels wait on their re-reads of earlier Q columns.
  if (nelem <= 256 * 2)
    k_block_ortho_df<2, 256, 3, 8><<<grid, 256, 0, st>>>(vecs, qdf, Vf, nc, bvol, nvec, fine, err, in32, out32);
  else if (nelem <= 512 * 3)
    k_block_ortho_df2<3, 512, 2, 2><<<grid, 512, 0, st>>>(vecs, qdf, Vf, nc, bvol, nvec, fine, err, in32, out32);
  else
    k_block_ortho_df<8, 256, 3, 8><<<grid, 256, 0, st>>>(vecs, qdf, Vf, nc, bvol, nvec, fine, err, in32, out32);
  WCMG_LAUNCH_CHECK();
}

void launch_block_ortho(double2* vecs, int Vf, int nc, int bvol, int nvec, bool fine, int* err, cudaStream_t st) {
  const int nelem = bvol * (nc / 2);
  if (nvec > 32) throw Error(-1, "block orthonormalisation supports nvec <= 32");
  if (nelem > 256 * 8) throw Error(-1, "aggregate too large for block orthonormalisation");
  const dim3 grid(Vf / bvol, 2);
  if (nelem <= 256 * 2) k_block_ortho<2><<<grid, 256, 0, st>>>(vecs, Vf, nc, bvol, nvec, fine, err);
  else if (nelem <= 256 * 4) k_block_ortho<4><<<grid, 256, 0, st>>>(vecs, Vf, nc, bvol, nvec, fine, err);
  else if (nelem <= 256 * 6) k_block_ortho<6><<<grid, 256, 0, st>>>(vecs, Vf, nc, bvol, nvec, fine, err);
  else k_block_ortho<8><<<grid, 256, 0, st>>>(vecs, Vf, nc, bvol, nvec, fine, err);
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
                                   cudaStream_t, int, const int*);                                              \
  template void launch_prolong<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, int, int, int, int, int, bool,      \
                                  cudaStream_t);                                                                \
  template void launch_make_columns<R>(cplx<R>*, const cplx<R>*, int, int, int, int, int, bool, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST

}  // namespace wcmg
