// Coarse-level kernels: the coarse Dirac operator as a nine-point stencil
// (Sec. 2.1 CoarsenedMatrix: Mdiag = self block, Mdir = hop block of one
// direction; Sec. 4: 9 stencil points), fused over all nine blocks:
//   y(x) = A_0(x) phi(x) + sum_mu [ A_{+mu}(x) phi(x + mu) + A_{-mu}(x) phi(x - mu) ]
// Per site the nine nb x nb blocks are stored as one row-major nb x ld matrix
// M(x) = [A_0 | A_{+x} | A_{-x} | ... | A_{-t}] (ld = 9 nb rounded up to 4), so
// y(x) = M(x) Phi(x) with Phi(x) the nine gathered neighbour vectors (staged in
// shared memory).  One CTA per coarse site streams M(x) with 16-byte loads; one
// warp per row, lanes split the row, warp-shuffle reduction.  The same kernel,
// with masked gathers, gives the block-interior and single-face parts that the
// Galerkin construction (CoarsenOperator) of the next level needs.
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace wcmg {

struct BlockInfoC { int b[4]; int bvol; };

__device__ __forceinline__ bool c_on_face(const BlockInfoC& bi, int s, int d) {
  int loc = s % bi.bvol;
  int l[4];
  l[0] = loc % bi.b[0]; loc /= bi.b[0];
  l[1] = loc % bi.b[1]; loc /= bi.b[1];
  l[2] = loc % bi.b[2];
  l[3] = loc / bi.b[2];
  const int mu = d >> 1;
  return (d & 1) ? (l[mu] == 0) : (l[mu] == bi.b[mu] - 1);
}

template <typename L, int VEC> struct alignas(16) LinkVec { L v[VEC]; };

// The gathered neighbour vectors sit in shared memory "transposed" by 16-byte link
// chunk: entry k = VEC g + v at v (ld / VEC) + g.  A lane that multiplies the VEC
// entries of link chunk g then reads, for each v, the word next to its neighbour
// lane's (no bank conflicts); in plain order the lanes' reads would be VEC entries
// apart, a VEC-way conflict for FP32 vectors and BF16 links.
template <int VEC>
__device__ __forceinline__ int phi_slot(int k, int ld) { return (k % VEC) * (ld / VEC) + k / VEC; }

template <typename L> __device__ __forceinline__ double2 link_to_c64(const L& l);
template <> __device__ __forceinline__ double2 link_to_c64<double2>(const double2& l) { return l; }
template <> __device__ __forceinline__ double2 link_to_c64<float2>(const float2& l) { return make_double2(l.x, l.y); }
template <> __device__ __forceinline__ double2 link_to_c64<bf16c>(const bf16c& l) {
  float2 f = __bfloat1622float2(l.v); return make_double2(f.x, f.y);
}
template <> __device__ __forceinline__ double2 link_to_c64<f16c>(const f16c& l) {
  float2 f = __half22float2(l.v); return make_double2(f.x, f.y);
}


template <typename R, typename L, int RR, int VEC>
__global__ void __launch_bounds__(512) k_coarse_apply(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                      const L* __restrict__ links, const int* __restrict__ nbr,
                                                      int Vc, int nb, int ld, int nrhs, int mode, int hopdir,
                                                      BlockInfoC bi, const unsigned char* __restrict__ par) {
  using T = cplx<R>;
  extern __shared__ unsigned char smem_raw[];
  T* phi = reinterpret_cast<T*>(smem_raw);  // [RR][ld]
  // grid.x = sites x row parts: CTA (site, part) computes rows [row0, row1) of y(site)
  const int parts = gridDim.x / Vc;
  const int site = blockIdx.x / parts, part = blockIdx.x % parts;
  const int rpc = (nb + parts - 1) / parts;
  const int row0 = part * rpc, row1 = min(nb, row0 + rpc);
  const int r0 = blockIdx.y * RR;
  const int K = 9 * nb;
  // link blocks this site needs: all nine for the full stencil; the self block and the
  // hops that stay inside the aggregate for the block interior; for a face hop only the
  // crossing block, and only on the face (a site off the face contributes nothing and
  // its output is never read: the face restriction reads face sites only)
  unsigned dmask = 0x1FFu;
  if (mode == ST_BLOCK_INTERIOR) {
    dmask = 1u;
    for (int d = 1; d < 9; ++d)
      if (!c_on_face(bi, site, d - 1)) dmask |= 1u << d;
  } else if (mode == ST_FACE_HOP) {
    dmask = c_on_face(bi, site, hopdir) ? 1u << (hopdir + 1) : 0u;
  }
  if (dmask == 0u) return;  // uniform over the CTA
  if (mode == ST_PARITY && par[site] != hopdir) {  // off-parity site: zero rows
    for (int idx = threadIdx.x; idx < RR * (row1 - row0); idx += blockDim.x) {
      const int r = idx / (row1 - row0), row = row0 + idx % (row1 - row0);
      if (r0 + r < nrhs) out[((long long)(r0 + r) * Vc + site) * nb + row] = czero<R>();
    }
    return;
  }
  const bool blockwise = (mode == ST_BLOCK_INTERIOR || mode == ST_FACE_HOP) && nb % VEC == 0;
  for (int idx = threadIdx.x; idx < RR * ld; idx += blockDim.x) {
    const int r = idx / ld, k = idx % ld;
    T v = czero<R>();
    if (k < K && r0 + r < nrhs) {
      const int d = k / nb, c = k % nb;
      bool inc = true;
      if (mode == ST_BLOCK_INTERIOR) inc = (d == 0) || !c_on_face(bi, site, d - 1);
      else if (mode == ST_FACE_HOP) inc = (d >= 1) && (d - 1 == hopdir) && c_on_face(bi, site, d - 1);
      if (inc) {
        const int n = d == 0 ? site : nbr[(d - 1) * Vc + site];
        v = in[((long long)(r0 + r) * Vc + n) * nb + c];
      }
    }
    phi[(idx / ld) * ld + phi_slot<VEC>(idx % ld, ld)] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = ld / VEC;
  for (int row = row0 + warp; row < row1; row += nw) {
    const L* lr = links + ((long long)site * nb + row) * ld;
    T acc[RR];
#pragma unroll
    for (int r = 0; r < RR; ++r) acc[r] = czero<R>();
    if (blockwise) {  // stream only the needed blocks of the row
      for (int d = 0; d < 9; ++d) {
        if (!((dmask >> d) & 1u)) continue;
        for (int k0 = d * nb + lane * VEC; k0 < (d + 1) * nb; k0 += 32 * VEC) {
          const LinkVec<L, VEC> lv = *reinterpret_cast<const LinkVec<L, VEC>*>(lr + k0);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const T a = link_load<L, R>(lv.v[v]);
#pragma unroll
            for (int r = 0; r < RR; ++r) cmac(acc[r], a, phi[r * ld + v * G + k0 / VEC]);
          }
        }
      }
    } else {
#pragma unroll 4
      for (int k0 = lane * VEC; k0 < ld; k0 += 32 * VEC) {
        const LinkVec<L, VEC> lv = *reinterpret_cast<const LinkVec<L, VEC>*>(lr + k0);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T a = link_load<L, R>(lv.v[v]);
#pragma unroll
          for (int r = 0; r < RR; ++r) cmac(acc[r], a, phi[r * ld + v * G + k0 / VEC]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RR; ++r) {
      const T s = warp_sum(acc[r]);
      if (lane == 0 && r0 + r < nrhs) out[((long long)(r0 + r) * Vc + site) * nb + row] = s;
    }
  }
}

// Masked coarse applies of the Galerkin construction (block interior, one face hop) with
// many fields, as one small complex GEMM per coarse site:
//   Y(x) [nb x nf] = sum over the blocks d the mask keeps at x of A_d(x) Phi_d(x),
// Phi_d(x) the nf input fields at the d-neighbour of x.  One CTA per (site, tile of up to
// 16 TN fields): each kept block A_d (nb x nb, rows padded by one entry so that the rows a
// warp reads fall in distinct banks) and Phi_d (nb x tile, transposed, padded likewise)
// are staged in shared memory, and a 16 x 16 thread grid accumulates a TM x TN register
// tile (rows tr + 16 i, fields tc + 16 j).  A site that keeps no block (a face hop off the
// face) returns at once; its output is never read.  Compared with the row-per-warp
// kernel this removes the warp-shuffle sum of every row and field.
template <typename R, typename L, int TM, int TN>
__global__ void __launch_bounds__(256) k_coarse_masked_gemm(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                            const L* __restrict__ links, const int* __restrict__ nbr,
                                                            int Vc, int nb, int ld, int nrhs, int mode, int hopdir,
                                                            BlockInfoC bi) {
  using T = cplx<R>;
  constexpr int NT = 16 * TN;
  extern __shared__ unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);  // [nb][nb + 1]
  T* Ps = As + nb * (nb + 1);                // [nb][NT + 1]
  const int site = blockIdx.x, c0 = blockIdx.y * NT;
  const int ncl = min(NT, nrhs - c0);
  unsigned dmask;
  if (mode == ST_BLOCK_INTERIOR) {
    dmask = 1u;
    for (int d = 1; d < 9; ++d)
      if (!c_on_face(bi, site, d - 1)) dmask |= 1u << d;
  } else {
    dmask = c_on_face(bi, site, hopdir) ? 1u << (hopdir + 1) : 0u;
  }
  if (dmask == 0u || ncl <= 0) return;  // uniform over the CTA
  const int tr = threadIdx.x & 15, tc = threadIdx.x >> 4;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = czero<R>();
  for (int d = 0; d < 9; ++d) {
    if (!((dmask >> d) & 1u)) continue;
    __syncthreads();  // the previous block's reads are done
    const L* lr = links + (long long)site * nb * ld + d * nb;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int a = idx / nb, b = idx - a * nb;
      As[a * (nb + 1) + b] = link_load<L, R>(lr[(long long)a * ld + b]);
    }
    const int n = d == 0 ? site : nbr[(d - 1) * Vc + site];
    for (int idx = threadIdx.x; idx < ncl * nb; idx += blockDim.x) {
      const int c = idx / nb, b = idx - c * nb;
      Ps[b * (NT + 1) + c] = in[((long long)(c0 + c) * Vc + n) * nb + b];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < nb; ++k) {
      T p[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) p[j] = Ps[k * (NT + 1) + tc + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int row = tr + 16 * i;
        if (row < nb) {
          const T a = As[row * (nb + 1) + k];
#pragma unroll
          for (int j = 0; j < TN; ++j) cmac(acc[i][j], a, p[j]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int row = tr + 16 * i, col = tc + 16 * j;
      if (row < nb && col < ncl) out[((long long)(c0 + col) * Vc + site) * nb + row] = acc[i][j];
    }
}

size_t coarse_masked_gemm_smem(int nb, int nrhs, int elem_bytes) {
  const int tn = (std::min(nrhs, 64) + 15) / 16;
  return (size_t)(nb * (nb + 1) + nb * (16 * tn + 1)) * elem_bytes;
}

template <typename R, typename L>
static void coarse_masked_gemm(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb, int nrhs,
                               int mode, int hopdir, cudaStream_t st) {
  BlockInfoC bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const int tm = (nb + 15) / 16, tn = (std::min(nrhs, 64) + 15) / 16;
  const size_t smem = coarse_masked_gemm_smem(nb, nrhs, (int)sizeof(cplx<R>));
  const dim3 grid((unsigned)g.V, (unsigned)((nrhs + 16 * tn - 1) / (16 * tn)));
  const int ld = links_ld(nb);
#define WCMG_MG(TM, TN)                                                                                      \
  do {                                                                                                       \
    auto kern = k_coarse_masked_gemm<R, L, TM, TN>;                                                          \
    if (smem > 48 * 1024) WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                         (int)smem));                                        \
    kern<<<grid, 256, smem, st>>>(out, in, links, g.nbr, g.V, nb, ld, nrhs, mode, hopdir, bi);                \
  } while (0)
#define WCMG_MGN(TM) \
  if (tn == 1) WCMG_MG(TM, 1); else if (tn == 2) WCMG_MG(TM, 2); else if (tn == 3) WCMG_MG(TM, 3); else WCMG_MG(TM, 4)
  if (tm == 1) { WCMG_MGN(1); }
  else if (tm == 2) { WCMG_MGN(2); }
  else if (tm == 3) { WCMG_MGN(3); }
  else { WCMG_MGN(4); }
#undef WCMG_MGN
#undef WCMG_MG
  WCMG_LAUNCH_CHECK();
}

// Single-rhs coarse apply.  One CTA per (site, block of rows): the nine
// neighbour vectors are gathered once into shared memory; each warp owns rows
// and loads RPW whole rows (NK 16-byte chunks per lane each) before reducing them;
// the first rows are requested before the gather and the barrier, so every warp has
// RPW rows (RPW x NK x 512 B) of the link stream in flight.  RPW = 2 keeps as many
// bytes in flight per warp for 4-byte (BF16 / FP16) links as RPW = 1 does for FP32.
template <typename R, typename L, int VEC, int NK, int RPW>
__global__ void __launch_bounds__(512) k_coarse_apply1(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                       const L* __restrict__ links, const int* __restrict__ nbr,
                                                       int Vc, int nb, int ld, int parts) {
  using T = cplx<R>;
  extern __shared__ unsigned char smem_raw[];
  T* phi = reinterpret_cast<T*>(smem_raw);  // [ld]
  const int site = blockIdx.x / parts, part = blockIdx.x % parts;
  const int rpc = (nb + parts - 1) / parts;
  const int row0 = part * rpc, row1 = min(nb, row0 + rpc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const L* base = links + (long long)site * nb * ld;
  LinkVec<L, VEC> cur[RPW][NK];
  auto load_rows = [&](int row) {
#pragma unroll
    for (int u = 0; u < RPW; ++u) {
      const int r = row + u * nw;
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        const int k0 = VEC * (lane + 32 * j);
        if (r < row1 && k0 < ld) cur[u][j] = *reinterpret_cast<const LinkVec<L, VEC>*>(base + (long long)r * ld + k0);
      }
    }
  };
  int row = row0 + warp;
  load_rows(row);
  const int K = 9 * nb;
  for (int idx = threadIdx.x; idx < ld; idx += blockDim.x) {
    T v = czero<R>();
    if (idx < K) {
      const int d = idx / nb, c = idx - d * nb;
      const int n = d == 0 ? site : nbr[(d - 1) * Vc + site];
      v = in[(long long)n * nb + c];
    }
    phi[phi_slot<VEC>(idx, ld)] = v;
  }
  __syncthreads();
  const int G = ld / VEC;
  for (; row < row1; row += RPW * nw) {
    if (row != row0 + warp) load_rows(row);
    T acc[RPW];
#pragma unroll
    for (int u = 0; u < RPW; ++u) acc[u] = czero<R>();
#pragma unroll
    for (int j = 0; j < NK; ++j) {
      const int k0 = VEC * (lane + 32 * j);
      if (k0 < ld) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T p = phi[v * G + k0 / VEC];
#pragma unroll
          for (int u = 0; u < RPW; ++u) cmac(acc[u], link_load<L, R>(cur[u][j].v[v]), p);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RPW; ++u) {
      const T a = warp_sum(acc[u]);
      if (lane == 0 && row + u * nw < row1) out[(long long)site * nb + row + u * nw] = a;
    }
  }
}

// One-rhs coarse apply from the five-block storage (kind 5).  D_c = P^dag D P inherits
// gamma5-hermiticity: gamma5 P = P sigma3 for the chirality-split basis (sigma3 = +1
// on a site's first Nvec basis vectors, -1 on the rest), so D_c^dag = sigma3 D_c
// sigma3, and since each fine hop and its reverse cross the same face, face by face
//   A_{-mu}(x) = sigma3 A_{+mu}(x - mu)^dag sigma3.
// Only M5(x) = [A_0 | A_{+x} | A_{+y} | A_{+z} | A_{+t}] is kept (row-major nb x ld5,
// ld5 = 5 nb rounded up to 4), 5/9 of the nine-block bytes:
//   y(x)_a = sum_k M5(x)_{ak} Phi5(x)_k + s_a sum_mu sum_b conj(A_{+mu}(x - mu)_{ba}) s_b phi(x - mu)_b.
// The forward part is the nine-block kernel's (one warp per row, 16-byte loads, RPW rows
// in flight, conflict-free gathered vectors) and runs first, so the link stream starts at
// once; each warp then joins the backward part, which reads the neighbours' forward
// blocks row by row as well: with VB (nb a multiple of the 16-byte chunk), thread
// t owns chunk g = t mod G of every row (G = nb / VEC chunks) and the rows t / G + k RG
// of all four blocks, accumulating the VEC outputs of its chunk privately; the RG partial
// vectors are then summed in a fixed order.  Otherwise thread (mu, a) walks column a of
// block mu.  Those blocks were streamed from HBM by the neighbours' own CTAs shortly
// before (sites go in storage order; the -t neighbour is one time slice back), so they
// mostly come from L2 and HBM sees about 5/9 of the nine-block bytes.
template <typename R, typename L, int VEC, int NK, int RPW, bool VB>
__global__ void __launch_bounds__(512) k_coarse_apply5(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                       const L* __restrict__ links5, const int* __restrict__ nbr,
                                                       int Vc, int nb, int ld5) {
  using T = cplx<R>;
  extern __shared__ unsigned char smem_raw[];
  T* phi = reinterpret_cast<T*>(smem_raw);  // [ld5] forward vectors (phi_slot order)
  T* phib = phi + ld5;                      // [4][nb] s_b phi(x - mu)_b
  T* yf = phib + 4 * nb;                    // [nb] forward part of y
  T* part = yf + nb;                        // VB: [RG][nb] backward partial sums; else [4][nb]
  const int site = blockIdx.x;
  const int half = nb >> 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const L* base = links5 + (long long)site * nb * ld5;
  LinkVec<L, VEC> cur[RPW][NK];
  auto load_rows = [&](int row) {
#pragma unroll
    for (int u = 0; u < RPW; ++u) {
      const int r = row + u * nw;
#pragma unroll
      for (int j = 0; j < NK; ++j) {
        const int k0 = VEC * (lane + 32 * j);
        if (r < nb && k0 < ld5) cur[u][j] = *reinterpret_cast<const LinkVec<L, VEC>*>(base + (long long)r * ld5 + k0);
      }
    }
  };
  int row = warp;
  load_rows(row);
  for (int idx = threadIdx.x; idx < ld5; idx += blockDim.x) {
    T v = czero<R>();
    if (idx < 5 * nb) {
      const int d = idx / nb, c = idx - d * nb;
      const int n = d == 0 ? site : nbr[(2 * (d - 1)) * Vc + site];  // +mu neighbour
      v = in[(long long)n * nb + c];
    }
    phi[phi_slot<VEC>(idx, ld5)] = v;
  }
  for (int idx = threadIdx.x; idx < 4 * nb; idx += blockDim.x) {
    const int mu = idx / nb, b = idx - mu * nb;
    const T v = in[(long long)nbr[(2 * mu + 1) * Vc + site] * nb + b];  // -mu neighbour
    phib[idx] = b < half ? v : -v;
  }
  __syncthreads();
  // forward part first (HBM stream; the first rows are already in flight), kept in yf
  const int G5 = ld5 / VEC;
  for (; row < nb; row += RPW * nw) {
    if (row != warp) load_rows(row);
    T acc[RPW];
#pragma unroll
    for (int u = 0; u < RPW; ++u) acc[u] = czero<R>();
#pragma unroll
    for (int j = 0; j < NK; ++j) {
      const int k0 = VEC * (lane + 32 * j);
      if (k0 < ld5) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const T p = phi[v * G5 + k0 / VEC];
#pragma unroll
          for (int u = 0; u < RPW; ++u) cmac(acc[u], link_load<L, R>(cur[u][j].v[v]), p);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < RPW; ++u) {
      const T a = warp_sum(acc[u]);
      const int r = row + u * nw;
      if (lane == 0 && r < nb) yf[r] = a;
    }
  }
  // backward part (mostly L2), overlapping the other warps' forward rows
  if constexpr (VB) {
    const int G = nb / VEC, RG = (int)blockDim.x / G;
    const int g = threadIdx.x % G, rg = threadIdx.x / G;
    if (rg < RG) {
      T acc[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[v] = czero<R>();
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        const int n = nbr[(2 * mu + 1) * Vc + site];
        const L* blk = links5 + (long long)n * nb * ld5 + (1 + mu) * nb + VEC * g;
        const T* pb = phib + mu * nb;
#pragma unroll 4
        for (int b = rg; b < nb; b += RG) {
          const LinkVec<L, VEC> w = *reinterpret_cast<const LinkVec<L, VEC>*>(blk + (long long)b * ld5);
          const T p = pb[b];
#pragma unroll
          for (int v = 0; v < VEC; ++v) cjmac(acc[v], link_load<L, R>(w.v[v]), p);
        }
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) part[rg * nb + VEC * g + v] = acc[v];
    }
    __syncthreads();
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      T sum = czero<R>();
      for (int r = 0; r < RG; ++r) sum += part[r * nb + a];
      out[(long long)site * nb + a] = yf[a] + (a < half ? sum : -sum);
    }
  } else {
    for (int t = threadIdx.x; t < 4 * nb; t += blockDim.x) {
      const int mu = t / nb, a = t - mu * nb;
      const int n = nbr[(2 * mu + 1) * Vc + site];
      const L* col = links5 + (long long)n * nb * ld5 + (1 + mu) * nb + a;
      const T* pb = phib + mu * nb;
      T acc = czero<R>();
#pragma unroll 8
      for (int b = 0; b < nb; ++b) cjmac(acc, link_load<L, R>(col[(long long)b * ld5]), pb[b]);
      part[t] = acc;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < nb; a += blockDim.x) {
      const T sum = part[a] + part[nb + a] + part[2 * nb + a] + part[3 * nb + a];
      out[(long long)site * nb + a] = yf[a] + (a < half ? sum : -sum);
    }
  }
}

// nine-block rows [A_0 | A_{+x} | A_{-x} | ... ] -> five-block rows [A_0 | A_{+x} | A_{+y} | A_{+z} | A_{+t}]
template <typename L>
__global__ void k_links_to_5(L* __restrict__ dst, const L* __restrict__ src, int Vc, int nb, int ld, int ld5) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)Vc * nb * ld5;
  if (idx >= total) return;
  const int k = (int)(idx % ld5);
  const long long row = idx / ld5;  // site * nb + a
  L v;
  memset(&v, 0, sizeof(L));
  if (k < 5 * nb) {
    const int d5 = k / nb, c = k - d5 * nb;
    const int d9 = d5 == 0 ? 0 : 2 * d5 - 1;
    v = src[row * ld + (long long)d9 * nb + c];
  }
  dst[idx] = v;
}

// Single-rhs coarse apply as a streaming pipeline (kind 3).  Persistent CTAs walk
// the work items (site, chunk of `cr` link rows) in the order blockIdx.x + k
// gridDim.x; thread 0 keeps `stages` bulk copies (cp.async.bulk of one contiguous
// chunk of the row-major link matrix each, completion counted on the stage's
// mbarrier) in flight ahead of the arithmetic, so the link stream never waits on a
// dependent load the way a CTA per site does.  When an item's site changes, the
// nine neighbour vectors are gathered into shared memory; each warp then reduces
// whole rows of the staged chunk (16-byte shared loads, warp-shuffle sum).  Every
// wait is bounded: a timeout sets *err = 3, waits (bounded) for the copies still
// in flight and ends the CTA.
constexpr int STREAM_MAX_STAGES = 8;

template <typename R, typename L>
__global__ void __launch_bounds__(512) k_coarse_apply1_stream(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                                              const L* __restrict__ links, const int* __restrict__ nbr,
                                                              int Vc, int nb, int ld, int cr, int stages,
                                                              int* __restrict__ err) {
  using T = cplx<R>;
  constexpr int VEC = 16 / sizeof(L);
  constexpr int PF = 4;  // gathered entries per thread kept in registers for the next site (ld <= PF x threads)
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STREAM_MAX_STAGES];
  const int phi_bytes = (ld * (int)sizeof(T) + 127) / 128 * 128;
  T* phi[2] = {reinterpret_cast<T*>(smem), reinterpret_cast<T*>(smem + phi_bytes)};  // [ld] each, zero padded
  const int stage_bytes = (cr * ld * (int)sizeof(L) + 127) / 128 * 128;
  unsigned char* stage0 = smem + 2 * phi_bytes;
  const int cps = (nb + cr - 1) / cr;  // chunks per site
  // this CTA's sites: blockIdx.x + k gridDim.x; chunk q = k cps + c of them
  const long long nsites = Vc > (int)blockIdx.x ? (Vc - 1 - (int)blockIdx.x) / gridDim.x + 1 : 0;
  const long long nq = nsites * cps;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    for (int q = 0; q < stages; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](long long q) {
    const int site = (int)(blockIdx.x + (q / cps) * gridDim.x), r0 = (int)(q % cps) * cr;
    const int rows = min(cr, nb - r0);
    const uint32_t bytes = (uint32_t)rows * ld * sizeof(L);
    uint64_t* bar = &full[q % stages];
    mbar_expect_tx(bar, bytes);
    tma_load_1d(stage0 + (q % stages) * stage_bytes, links + ((long long)site * nb + r0) * ld, bytes, bar);
  };
  auto gather = [&](int site, T (&v)[PF]) {
#pragma unroll
    for (int p = 0; p < PF; ++p) {
      const int i = threadIdx.x + p * blockDim.x;
      v[p] = czero<R>();
      if (i < 9 * nb) {
        const int d = i / nb, c = i - d * nb;
        v[p] = in[(long long)(d == 0 ? site : nbr[(d - 1) * Vc + site]) * nb + c];
      }
    }
  };
  auto store = [&](T* dst, const T (&v)[PF]) {
#pragma unroll
    for (int p = 0; p < PF; ++p) {
      const int i = threadIdx.x + p * blockDim.x;
      if (i < ld) dst[phi_slot<VEC>(i, ld)] = v[p];
    }
  };
  if (threadIdx.x == 0)
    for (long long q = 0; q < stages && q < nq; ++q) issue(q);
  T pf[PF];
  if (nsites > 0) {
    gather((int)blockIdx.x, pf);
    store(phi[0], pf);
  }
  __syncthreads();
  long long q = 0;
  bool ok = true;
  for (long long k = 0; k < nsites && ok; ++k) {
    const int site = (int)(blockIdx.x + k * gridDim.x);
    const T* ph = phi[k & 1];
    if (k + 1 < nsites) gather((int)(blockIdx.x + (k + 1) * gridDim.x), pf);  // in flight during this site
    for (int c = 0; c < cps; ++c, ++q) {
      const int r0 = c * cr, rows = min(cr, nb - r0);
      const int s = (int)(q % stages);
      // one thread polls the barrier; the CTA barrier then orders the copied data for all
      const int good = threadIdx.x != 0 || mbar_wait_bounded(&full[s], (uint32_t)((q / stages) & 1)) ? 1 : 0;
      if (!__syncthreads_and(good)) {
        ok = false;
        break;
      }
      const L* chunk = reinterpret_cast<const L*>(stage0 + s * stage_bytes);
      for (int row = warp; row < rows; row += nw) {
        const L* lr = chunk + row * ld;
        T acc = czero<R>();
        for (int g = lane; g * VEC < ld; g += 32) {
          const LinkVec<L, VEC> lv = *reinterpret_cast<const LinkVec<L, VEC>*>(lr + g * VEC);
#pragma unroll
          for (int v = 0; v < VEC; ++v) cmac(acc, link_load<L, R>(lv.v[v]), ph[v * (ld / VEC) + g]);
        }
        acc = warp_sum(acc);
        if (lane == 0) out[(long long)site * nb + r0 + row] = acc;
      }
      __syncthreads();  // stage s consumed
      if (threadIdx.x == 0 && q + stages < nq) issue(q + stages);
    }
    if (ok && k + 1 < nsites) {
      store(phi[(k + 1) & 1], pf);
      __syncthreads();
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicExch(err, 3);
    for (long long r = q; r < q + stages && r < nq; ++r)  // copies still in flight
      mbar_wait_bounded(&full[r % stages], (uint32_t)((r / stages) & 1));
  }
}

// Multi-rhs coarse apply on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulation in TMEM).  Per coarse site x the nine blocks form
// Y = M(x) Phi(x), M: nb x 9 nb complex, Phi: 9 nb x N complex.  Real form along K
// (k' = 2 k + 0 / + 1): A is M as stored, its BF16 (Re, Im) pairs side by side,
//   A[a][2k] = Re M[a][k],  A[a][2k+1] = Im M[a][k]              (rows a < nb)
// and the complex product goes into B, two columns per rhs n:
//   B[n][2k] = Re Phi[k][n],  B[n][2k+1] = -Im Phi[k][n]         (D[a][n] = Re Y[a][n])
//   B[N+n][2k] = Im Phi[k][n], B[N+n][2k+1] = Re Phi[k][n]       (D[a][N+n] = Im Y[a][n])
// M_mma = 128 (rows nb .. 127 zero), N_mma = 2 N.  A chunk of A is then a plain
// copy of 16-byte groups of the link rows (no conversion).  One CTA (4 warps) per
// (site, tile of <= 64 rhs).  K is walked in chunks of 64: the chunk is read from
// global memory into registers one step ahead and stored into one of two
// shared-memory stages in the no-swizzle K-major core-matrix layout, and one
// thread issues four K = 16 MMAs and commits them to the stage's mbarrier.  Every
// wait is bounded; a timeout sets *err = 3, frees the TMEM and ends the CTA.
constexpr int MMA_M = 128, MMA_KC = 64, MMA_LBO = 128, MMA_SBO = (MMA_KC / 8) * 128;
constexpr int MMA_AQ = 4, MMA_BE = 16;  // per-thread staging: nb <= 64 rows x 8 groups, rhs tile <= 64

__device__ __forceinline__ int mma_off(int row, int k) {
  return (row >> 3) * MMA_SBO + (k >> 3) * MMA_LBO + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <typename L>
__global__ void __launch_bounds__(128) k_coarse_apply_mma(float2* __restrict__ out, const float2* __restrict__ in,
                                                          const L* __restrict__ links, const int* __restrict__ nbr,
                                                          int Vc, int nb, int ld, int nrhs, int ntile, int tmem_cols,
                                                          int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int nsite[9];
  static_assert(sizeof(L) == 4, "links: one BF16 (Re, Im) pair per entry");
  const int a_bytes = MMA_M * MMA_KC * 2, stage_bytes = a_bytes + 2 * ntile * MMA_KC * 2;
  const int site = blockIdx.x, r0 = blockIdx.y * ntile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Kc = 9 * nb, nchunks = (2 * Kc + MMA_KC - 1) / MMA_KC;
  const int nvalid = min(ntile, nrhs - r0);
  for (int i = tid; i < 2 * stage_bytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 9) nsite[tid] = tid == 0 ? site : nbr[(tid - 1) * Vc + site];
  if (warp == 0) tmem_alloc(&tmem_base, tmem_cols);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = umma_idesc_bf16(MMA_M, 2 * ntile);
  const L* lsite = links + (long long)site * nb * ld;
  const uint32_t* lwords = reinterpret_cast<const uint32_t*>(lsite);
  uint4 ra[MMA_AQ];
  float2 rb[MMA_BE];
  auto load_chunk = [&](int c) {
    const int kc0 = c * (MMA_KC / 2);
    // A: group g of row a = link entries kc0 + 4 g .. + 3 (16 bytes; ld and the row
    // starts are multiples of 4 entries), entries at or beyond 9 nb read as 0
#pragma unroll
    for (int q = 0; q < MMA_AQ; ++q) {
      const int e = tid + 128 * q;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (e < nb * 8) {
        const int a = e >> 3, k = kc0 + 4 * (e & 7);
        const long long o = (long long)a * ld + k;
        if (k + 3 < Kc) {
          v = *reinterpret_cast<const uint4*>(lsite + o);
        } else {
          if (k < Kc) v.x = lwords[o];
          if (k + 1 < Kc) v.y = lwords[o + 1];
          if (k + 2 < Kc) v.z = lwords[o + 2];
        }
      }
      ra[q] = v;
    }
#pragma unroll
    for (int q = 0; q < MMA_BE; ++q) {
      const int e = tid + 128 * q;
      float2 v = make_float2(0.f, 0.f);
      if (e < ntile * (MMA_KC / 2)) {
        const int n = e >> 5, k = kc0 + (e & 31);
        if (n < nvalid && k < Kc) {
          const int d = k / nb, cc = k - d * nb;
          v = in[((long long)(r0 + n) * Vc + nsite[d]) * nb + cc];
        }
      }
      rb[q] = v;
    }
  };
  auto store_chunk = [&](int s) {
    unsigned char* A = smem + s * stage_bytes;
    unsigned char* B = A + a_bytes;
#pragma unroll
    for (int q = 0; q < MMA_AQ; ++q) {
      const int e = tid + 128 * q;
      if (e < nb * 8) *reinterpret_cast<uint4*>(A + mma_off(e >> 3, 8 * (e & 7))) = ra[q];
    }
#pragma unroll
    for (int q = 0; q < MMA_BE; ++q) {
      const int e = tid + 128 * q;
      if (e < ntile * (MMA_KC / 2)) {
        const int n = e >> 5, kk = 2 * (e & 31);
        *reinterpret_cast<uint32_t*>(B + mma_off(n, kk)) = pack_bf16x2(rb[q].x, -rb[q].y);
        *reinterpret_cast<uint32_t*>(B + mma_off(ntile + n, kk)) = pack_bf16x2(rb[q].y, rb[q].x);
      }
    }
  };
  bool ok = true;
  load_chunk(0);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    if (c >= 2) {  // the MMAs of chunk c - 2 read this stage
      const int good = mbar_wait_bounded(&bar[s], (uint32_t)(((c - 2) >> 1) & 1)) ? 1 : 0;
      if (!__syncthreads_and(good)) { ok = false; break; }
    }
    store_chunk(s);
    if (c + 1 < nchunks) load_chunk(c + 1);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(smem + s * stage_bytes), b0 = a0 + a_bytes;
#pragma unroll
      for (int q = 0; q < MMA_KC / 16; ++q)
        umma_bf16(tmem, umma_desc(a0 + q * 2 * MMA_LBO, MMA_LBO, MMA_SBO),
                  umma_desc(b0 + q * 2 * MMA_LBO, MMA_LBO, MMA_SBO), idesc, (c > 0 || q > 0) ? 1u : 0u);
      umma_commit(&bar[s]);
    }
  }
  if (ok) {
    const int cl = nchunks - 1;
    const int good = mbar_wait_bounded(&bar[cl & 1], (uint32_t)((cl >> 1) & 1)) ? 1 : 0;
    ok = __syncthreads_and(good) != 0;
  }
  if (ok) {
    tc_fence_after();
    const int m = 32 * warp + lane;
    float* o = reinterpret_cast<float*>(out);
    // column np < ntile: Re Y[m][np]; np >= ntile: Im Y[m][np - ntile]
    for (int j = 0; j < 2 * ntile / 16; ++j) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * j, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int np = 16 * j + i, part = np < ntile ? 0 : 1, n = np - part * ntile;
        if (n < nvalid && m < nb) o[2 * (((long long)(r0 + n) * Vc + site) * nb + m) + part] = v[i];
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 3);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// Multi-rhs coarse apply on tcgen05 with every operand moved by bulk copies
// (kind 4).  Per coarse site x: Y = M(x) Phi(x) in the real form of the kind-2
// kernel (A = the links' BF16 (Re, Im) pairs along K, the complex product in B).
// Operands are pre-arranged in global memory in the no-swizzle K-major layout of
// the MMA, so that one contiguous bulk copy fills an operand of a neighbour block:
//   A (links, "MMA copy"): [site][d][g][a][8 BF16]: group g of row a of block A_d is
//     the 16 bytes of link entries 4 g .. 4 g + 3 (nb / 4 groups, nb rows);
//   B (built by k_mma_bprep for each apply): [y][tile][g][j][8 BF16] with rows
//     j < N: (Re phi, -Im phi) of rhs tile N + j at site y, j >= N: (Im phi, Re phi).
// In shared memory a stage then holds A_d (nb rows x 2 nb K) and B (2 N rows x 2 nb
// K) with leading byte offsets 16 nb and 32 N; an MMA of M rows (64 or 128; rows
// beyond nb read neighbouring data and are never stored) and N_mma = 2 N runs over
// K = 16 per instruction.  Warp roles, persistent over (site, tile) items: warp 0
// issues the bulk copies into a ring of stages (full barriers with transaction
// counts), warp 1 allocates TMEM and issues the MMAs (committing each stage back to
// its empty barrier and each finished item to an accumulator barrier; two TMEM
// accumulators alternate), warps 2-5 read the accumulator of the previous item and
// store it while the next one is being formed.  Every wait is bounded: a timeout
// sets *err = 3; the CTA then waits (bounded) for its copies and MMAs in flight,
// frees its TMEM and ends.
constexpr int MMA4_MAX_STAGES = 8;

__global__ void k_mma_bprep(uint4* __restrict__ bp, const float2* __restrict__ in, int Vc, int nb, int nrhs,
                            int ntile, int ntiles) {
  // one thread per 16-byte group: (y, tile, g, j)
  const int kg = nb / 4, rows = 2 * ntile;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)Vc * ntiles * kg * rows;
  if (idx >= total) return;
  const int j = (int)(idx % rows);
  const int g = (int)((idx / rows) % kg);
  const long long yt = idx / ((long long)rows * kg);
  const int t = (int)(yt % ntiles), y = (int)(yt / ntiles);
  const int n = t * ntile + (j < ntile ? j : j - ntile);
  uint4 w = make_uint4(0, 0, 0, 0);
  if (n < nrhs) {
    const float4* src = reinterpret_cast<const float4*>(in + ((long long)n * Vc + y) * nb + 4 * g);
    const float4 a = src[0], b = src[1];  // phi entries 4 g .. 4 g + 3
    if (j < ntile) {
      w.x = pack_bf16x2(a.x, -a.y); w.y = pack_bf16x2(a.z, -a.w);
      w.z = pack_bf16x2(b.x, -b.y); w.w = pack_bf16x2(b.z, -b.w);
    } else {
      w.x = pack_bf16x2(a.y, a.x); w.y = pack_bf16x2(a.w, a.z);
      w.z = pack_bf16x2(b.y, b.x); w.w = pack_bf16x2(b.w, b.z);
    }
  }
  bp[idx] = w;
}

// links (row-major nb x ld per site, BF16 pairs) -> the MMA copy [site][d][g][a]
__global__ void k_links_to_mma(uint4* __restrict__ dst, const uint4* __restrict__ src, int Vc, int nb, int ld) {
  const int kg = nb / 4;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long total = (long long)Vc * 9 * kg * nb;
  if (idx >= total) return;
  const int a = (int)(idx % nb);
  const int g = (int)((idx / nb) % kg);
  const int d = (int)((idx / ((long long)nb * kg)) % 9);
  const long long site = idx / ((long long)nb * kg * 9);
  dst[idx] = src[((site * nb + a) * ld + d * nb + 4 * g) / 4];
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 32 lanes x 8 columns of FP32 from TMEM
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

template <int MM>
__global__ void __launch_bounds__(192, 1) k_coarse_apply_mma4(float2* __restrict__ out, const uint4* __restrict__ amma,
                                                              const uint4* __restrict__ bpre,
                                                              const int* __restrict__ nbr, int Vc, int nb, int nrhs,
                                                              int ntile, int ntiles, int stages,
                                                              int acc_cols, int nacc, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[MMA4_MAX_STAGES], empty[MMA4_MAX_STAGES], tfull[2], tempty[2], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kg = nb / 4, rows_b = 2 * ntile;
  const uint32_t a_bytes = (uint32_t)kg * nb * 16, b_bytes = (uint32_t)kg * rows_b * 16;
  const uint32_t a_alloc = (a_bytes + (uint32_t)(MM > nb ? MM - nb : 0) * 16 + 1023) / 1024 * 1024;
  const uint32_t stage_bytes = a_alloc + (b_bytes + 1023) / 1024 * 1024;
  const long long items = (long long)Vc * ntiles;
  const long long limit = 1LL << 26;
  if (threadIdx.x == 0) {
    for (int q = 0; q < stages; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&tfull[q], 1);
      mbar_init(&tempty[q], 128);
    }
    mbar_init(&fin, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_base, nacc * acc_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t s0 = smem_u32(smem);
  auto fail = [&]() {
    *(volatile int*)&abort_flag = 1;
    atomicExch(err, 3);
  };
  long long issued = 0;  // producer: chunks whose copies were issued
  if (warp == 0) {
    if (lane == 0) {
      long long c = 0;
      // neighbour indices of the next item, loaded one item ahead so that no copy waits
      // on a dependent global load
      int ny[8];
      auto load_nbr = [&](long long it) {
        const int site = (int)(it / ntiles);
#pragma unroll
        for (int d = 0; d < 8; ++d) ny[d] = it < items ? nbr[d * Vc + site] : 0;
      };
      load_nbr(blockIdx.x);
      for (long long it = blockIdx.x; it < items && !*(volatile int*)&abort_flag; it += gridDim.x) {
        const int site = (int)(it / ntiles), t = (int)(it % ntiles);
        int cur[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) cur[d] = ny[d];
        load_nbr(it + gridDim.x);
        for (int d = 0; d < 9; ++d, ++c) {
          const int s = (int)(c % stages);
          if (!mbar_wait_bounded(&empty[s], (uint32_t)(((c / stages) & 1) ^ 1), limit)) { fail(); break; }
          const int y = d == 0 ? site : cur[d - 1];
          unsigned char* st = smem + (size_t)s * stage_bytes;
          mbar_expect_tx(&full[s], a_bytes + b_bytes);
          tma_load_1d(st, amma + ((long long)site * 9 + d) * kg * nb, a_bytes, &full[s]);
          tma_load_1d(st + a_alloc, bpre + ((long long)y * ntiles + t) * kg * rows_b, b_bytes, &full[s]);
          issued = c + 1;
        }
        if (*(volatile int*)&abort_flag) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_bf16(MM, rows_b);
      long long c = 0, i = 0;
      bool ok = true;
      for (long long it = blockIdx.x; it < items && ok; it += gridDim.x, ++i) {
        const int tb = (int)(i % nacc);
        if (!mbar_wait_bounded(&tempty[tb], (uint32_t)(((i / nacc) & 1) ^ 1), limit)) { fail(); ok = false; break; }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(tb * acc_cols);
        for (int d = 0; d < 9; ++d, ++c) {
          const int s = (int)(c % stages);
          if (!mbar_wait_bounded(&full[s], (uint32_t)((c / stages) & 1), limit)) { fail(); ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = s0 + (uint32_t)s * stage_bytes, b0 = a0 + a_alloc;
          for (int q = 0; q < kg / 2; ++q)
            umma_bf16(dt, umma_desc(a0 + (uint32_t)q * 2 * nb * 16, (uint32_t)nb * 16, 128),
                      umma_desc(b0 + (uint32_t)q * 2 * rows_b * 16, (uint32_t)rows_b * 16, 128), idesc,
                      (d > 0 || q > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
        }
        if (!ok) break;
        umma_commit(&tfull[tb]);
      }
      umma_commit(&fin);  // every MMA issued by this CTA has completed once fin flips
      if (!mbar_wait_bounded(&fin, 0, limit)) fail();
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; row m of D sits in lane m (M = 128)
    // or lane 32 (m / 16) + m % 16 (M = 64)
    const int quad = warp & 3;
    const int m = MM == 128 ? 32 * quad + lane : (lane < 16 ? 16 * quad + lane : nb);
    long long i = 0;
    for (long long it = blockIdx.x; it < items; it += gridDim.x, ++i) {
      const int tb = (int)(i % nacc);
      // one lane per warp polls the accumulator barrier, the others wait at the warp barrier
      int good = lane != 0 || mbar_wait_bounded(&tfull[tb], (uint32_t)((i / nacc) & 1), limit) ? 1 : 0;
      good = __shfl_sync(0xffffffffu, good, 0);
      if (!good || *(volatile int*)&abort_flag) {
        if (!good) fail();
        break;
      }
      tc_fence_after();
      const int site = (int)(it / ntiles), t = (int)(it % ntiles);
      const uint32_t dt = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(tb * acc_cols);
      for (int j0 = 0; j0 < ntile; j0 += 8) {
        float re[8], im[8];
        tmem_ld8(dt + j0, re);
        tmem_ld8(dt + ntile + j0, im);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = t * ntile + j0 + q;
          if (m < nb && j0 + q < ntile && n < nrhs) out[((long long)n * Vc + site) * nb + m] = make_float2(re[q], im[q]);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[tb]);
    }
  }
  __syncthreads();
  if (warp == 0 && lane == 0 && *(volatile int*)&abort_flag) {
    // copies still in flight land before the CTA's shared memory is released
    for (long long q = issued - stages; q < issued; ++q)
      if (q >= 0) mbar_wait_bounded(&full[q % stages], (uint32_t)((q / stages) & 1), limit);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, nacc * acc_cols);
}

// Self-test of the bounded waits: one thread waits, at most `polls` polls, on the first
// phase of an mbarrier that nothing arrives on, so the wait gives up and the thread sets
// *err = 3 the way every bounded wait of the library does.  Nothing else is in flight
// (no copies, no TMEM), so the kernel ends normally and the context stays usable.
__global__ void k_wait_selftest(int* __restrict__ err, long long polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, polls)) atomicExch(err, 3);
}
void launch_wait_selftest(int* err, long long polls, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, polls);
  WCMG_LAUNCH_CHECK();
}

template <typename L> struct VecOf { static constexpr int v = 16 / sizeof(L); };

// ---------------- even-odd coarsest solve: self-block inverses ----------------
template <typename L>
__global__ void k_self_invert(double2* __restrict__ inv, const L* __restrict__ links, int nb, int ld,
                              int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* M = reinterpret_cast<double2*>(smem_raw);  // [nb][2 nb]: [A_0 | 1]
  __shared__ int piv;
  const int site = blockIdx.x, w = 2 * nb;
  for (int idx = threadIdx.x; idx < nb * w; idx += blockDim.x) {
    const int i = idx / w, j = idx % w;
    M[idx] = j < nb ? link_to_c64<L>(links[((long long)site * nb + i) * ld + j]) : make_double2(j - nb == i ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {  // partial pivoting: the largest |entry| of column k at or below row k
      int best = k;
      double bv = -1.0;
      for (int i = k; i < nb; ++i) {
        const double v = cnorm2(M[i * w + k]);
        if (v > bv) { bv = v; best = i; }
      }
      piv = best;
      if (!(bv > 0.0) || !isfinite(bv)) *err = 1;
    }
    __syncthreads();
    const int p = piv;
    if (p != k)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double2 t = M[k * w + j];
        M[k * w + j] = M[p * w + j];
        M[p * w + j] = t;
      }
    __syncthreads();
    const double2 d = M[k * w + k];
    const double dn = cnorm2(d);
    const double2 dinv = dn > 0.0 ? make_double2(d.x / dn, -d.y / dn) : make_double2(0.0, 0.0);
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) M[k * w + j] = cmul(dinv, M[k * w + j]);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nb * w; idx += blockDim.x) {
      const int i = idx / w, j = idx % w;
      if (i != k) cnmac(M[idx], M[i * w + k], M[k * w + j]);
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx % nb;
    inv[(long long)site * nb * nb + idx] = M[i * w + nb + j];
  }
}

template <typename L>
void launch_self_invert(double2* inv, const L* links, int Vc, int nb, int* err, cudaStream_t st) {
  const size_t smem = (size_t)nb * 2 * nb * sizeof(double2);
  auto kern = k_self_invert<L>;
  WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<Vc, 256, smem, st>>>(inv, links, nb, links_ld(nb), err);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_blockinv_apply(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in,
                                 const cplx<R>* __restrict__ inv, const unsigned char* __restrict__ par, int p, int Vc,
                                 int nb) {
  const int site = blockIdx.x, r = blockIdx.y;
  const cplx<R>* x = in + ((long long)r * Vc + site) * nb;
  cplx<R>* y = out + ((long long)r * Vc + site) * nb;
  const bool on = par[site] == p;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    cplx<R> acc = czero<R>();
    if (on) {
      const cplx<R>* row = inv + ((long long)site * nb + i) * nb;
      for (int j = 0; j < nb; ++j) cmac(acc, row[j], x[j]);
    }
    y[i] = acc;
  }
}

template <typename R>
void launch_blockinv_apply(cplx<R>* out, const cplx<R>* in, const cplx<R>* inv, const unsigned char* par, int p,
                           int Vc, int nb, int nrhs, cudaStream_t st) {
  k_blockinv_apply<R><<<dim3(Vc, nrhs), 64, 0, st>>>(out, in, inv, par, p, Vc, nb);
  WCMG_LAUNCH_CHECK();
}

template <typename R>
__global__ void k_parity_axpy(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ a, const cplx<R>* __restrict__ b,
                              R beta, const unsigned char* __restrict__ par, int p, int Vc, int nb, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int site = (int)((i / nb) % Vc);
  out[i] = par[site] == p ? a[i] + beta * b[i] : czero<R>();
}

template <typename R>
void launch_parity_axpy(cplx<R>* out, const cplx<R>* a, const cplx<R>* b, double beta, const unsigned char* par, int p,
                        int Vc, int nb, int nrhs, cudaStream_t st) {
  const long long n = (long long)nrhs * Vc * nb;
  k_parity_axpy<R><<<nblk(n, 256), 256, 0, st>>>(out, a, b, (R)beta, par, p, Vc, nb, n);
  WCMG_LAUNCH_CHECK();
}

template void launch_self_invert<double2>(double2*, const double2*, int, int, int*, cudaStream_t);
template void launch_self_invert<float2>(double2*, const float2*, int, int, int*, cudaStream_t);
#define WCMG_INST_EO(R)                                                                                         \
  template void launch_blockinv_apply<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const unsigned char*, int, int, \
                                         int, int, cudaStream_t);                                               \
  template void launch_parity_axpy<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, double, const unsigned char*, int, \
                                      int, int, int, cudaStream_t);
WCMG_INST_EO(double)
WCMG_INST_EO(float)
#undef WCMG_INST_EO

template <typename R, typename L, int RR>
static void coarse_apply_rr(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb, int nrhs,
                            int mode, int hopdir, int parts, cudaStream_t st) {
  constexpr int VEC = VecOf<L>::v;
  const int ld = links_ld(nb);
  BlockInfoC bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const size_t smem = (size_t)RR * ld * sizeof(cplx<R>);
  auto kern = k_coarse_apply<R, L, RR, VEC>;
  if (smem > 48 * 1024) WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long ncta_y = (nrhs + RR - 1) / RR;
  if (parts <= 0) {
    // enough CTAs to fill every SM several times over: split the rows of a site
    parts = 1;
    const long long want = 6LL * 152;
    while (parts < nb / 4 && (long long)g.V * parts * ncta_y < want) parts *= 2;
  }
  const int rpc = (nb + parts - 1) / parts;
  const int rpw = (rpc + 15) / 16;  // rows per warp, at most 16 warps
  const int threads = std::max(64, 32 * ((rpc + rpw - 1) / rpw));
  if (mode == ST_PARITY && !g.par) throw Error(-1, "coarse apply: parity mode needs the site parities");
  kern<<<dim3(g.V * parts, ncta_y), threads, smem, st>>>(out, in, links, g.nbr, g.V, nb, ld, nrhs, mode, hopdir,
                                                          bi, g.par);
  WCMG_LAUNCH_CHECK();
}

template <typename R, typename L>
static void coarse_apply1(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb, int parts,
                          int threads, int rpw, cudaStream_t st) {
  constexpr int VEC = VecOf<L>::v;
  const int ld = links_ld(nb);
  const int nk = (ld + 32 * VEC - 1) / (32 * VEC);
  const size_t smem = (size_t)ld * sizeof(cplx<R>);
  const unsigned grid = (unsigned)(g.V * parts);
#define WCMG_C1(NKV, RP) \
  k_coarse_apply1<R, L, VEC, NKV, RP><<<grid, threads, smem, st>>>(out, in, links, g.nbr, g.V, nb, ld, parts)
#define WCMG_C1R(NKV) \
  if (rpw == 2) WCMG_C1(NKV, 2); else WCMG_C1(NKV, 1)
  if (nk <= 4) { WCMG_C1R(4); }
  else if (nk <= 8) { WCMG_C1R(8); }
  else if (nk <= 12) { WCMG_C1(12, 1); }
  else if (nk <= 18) { WCMG_C1(18, 1); }
  else throw Error(-1, "coarse apply: nbasis too large");
#undef WCMG_C1R
#undef WCMG_C1
  WCMG_LAUNCH_CHECK();
}

template <typename R, typename L>
static void coarse_apply5(cplx<R>* out, const cplx<R>* in, const L* links5, const LevelGeom& g, int nb, int threads,
                          int rpw, cudaStream_t st) {
  constexpr int VEC = VecOf<L>::v;
  const int ld5 = links5_ld(nb);
  const int nk = (ld5 + 32 * VEC - 1) / (32 * VEC);
  const bool vb = nb % VEC == 0 && nb / VEC <= threads;
  const int rg = vb ? threads / (nb / VEC) : 4;
  const size_t smem = (size_t)(ld5 + 5 * nb + (size_t)rg * nb) * sizeof(cplx<R>);
  const unsigned grid = (unsigned)g.V;
#define WCMG_C5(NKV, RP, VB) \
  k_coarse_apply5<R, L, VEC, NKV, RP, VB><<<grid, threads, smem, st>>>(out, in, links5, g.nbr, g.V, nb, ld5)
#define WCMG_C5V(NKV, RP) \
  if (vb) WCMG_C5(NKV, RP, true); else WCMG_C5(NKV, RP, false)
#define WCMG_C5R(NKV) \
  if (rpw == 2) { WCMG_C5V(NKV, 2); } else { WCMG_C5V(NKV, 1); }
  if (smem > 48 * 1024) throw Error(-1, "coarse apply: five-block tile needs too much shared memory");
  if (nk <= 2) { WCMG_C5R(2); }
  else if (nk <= 4) { WCMG_C5R(4); }
  else if (nk <= 8) { WCMG_C5V(8, 1); }
  else if (nk <= 12) { WCMG_C5V(12, 1); }
  else throw Error(-1, "coarse apply: nbasis too large for the five-block kernel");
#undef WCMG_C5R
#undef WCMG_C5V
#undef WCMG_C5
  WCMG_LAUNCH_CHECK();
}

template <typename L>
void launch_links_to_5(L* dst, const L* src, int Vc, int nb, cudaStream_t st) {
  const long long total = (long long)Vc * nb * links5_ld(nb);
  k_links_to_5<L><<<nblk(total, 256), 256, 0, st>>>(dst, src, Vc, nb, links_ld(nb), links5_ld(nb));
  WCMG_LAUNCH_CHECK();
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    WCMG_CUDA(cudaGetDevice(&dev));
    WCMG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

// Resident CTAs per SM of a kernel launched with `threads` threads and `smem` bytes of
// dynamic shared memory, from the SM's own limits (shared memory with the maximum
// carveout, threads, registers).  The occupancy calculator was seen to answer 1 where
// two CTAs of 80 KB fit the 228 KB of an SM, so the limits are computed here.
static int blocks_per_sm(const void* kern, int threads, size_t smem) {
  WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  cudaFuncAttributes fa;
  WCMG_CUDA(cudaFuncGetAttributes(&fa, kern));
  int dev = 0, smem_sm = 0, reserved = 0, thr_sm = 0, regs_sm = 0;
  WCMG_CUDA(cudaGetDevice(&dev));
  WCMG_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  WCMG_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  WCMG_CUDA(cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
  WCMG_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  const size_t per_cta = smem + fa.sharedSizeBytes + (size_t)reserved;
  const int warps = (threads + 31) / 32;
  const int regs_warp = (std::max(fa.numRegs, 1) + 7) / 8 * 8 * 32;
  const int by_smem = (int)((size_t)smem_sm / per_cta);
  const int by_threads = thr_sm / (warps * 32);
  const int by_regs = regs_sm / (regs_warp * warps);
  return std::min(by_smem, std::min(by_threads, by_regs));
}

size_t coarse_stream_smem(int nb, int cr, int stages, int vec_bytes, int link_bytes) {
  const int ld = links_ld(nb);
  return 2 * ((size_t)(ld * vec_bytes + 127) / 128 * 128) + (size_t)stages * ((cr * ld * link_bytes + 127) / 128 * 128);
}

template <typename R, typename L>
static void coarse_apply1_stream(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb,
                                 int threads, int cr, int stages, int* err, cudaStream_t st) {
  const int ld = links_ld(nb);
  const size_t smem = coarse_stream_smem(nb, cr, stages, sizeof(cplx<R>), sizeof(L));
  auto kern = k_coarse_apply1_stream<R, L>;
  WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int per_sm = blocks_per_sm((const void*)kern, threads, smem);
  if (per_sm < 1) throw Error(-1, "coarse apply: streaming tile does not fit on an SM");
  if (ld > 4 * threads) throw Error(-1, "coarse apply: streaming tile needs more threads for this nbasis");
  const int grid = (int)std::min<long long>(g.V, (long long)sm_count() * per_sm);
  kern<<<grid, threads, smem, st>>>(out, in, links, g.nbr, g.V, nb, ld, cr, stages, err);
  WCMG_LAUNCH_CHECK();
}

template <typename L>
static void coarse_apply_mma(float2* out, const float2* in, const L* links, const LevelGeom& g, int nb, int nrhs,
                             int ntile, int* err, cudaStream_t st) {
  const int ld = links_ld(nb);
  const int tmem_cols = ntile <= 16 ? 32 : (ntile <= 32 ? 64 : 128);  // 2 ntile FP32 columns
  const size_t smem = 2 * ((size_t)MMA_M * MMA_KC * 2 + (size_t)2 * ntile * MMA_KC * 2);
  auto kern = k_coarse_apply_mma<L>;
  WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<dim3(g.V, (nrhs + ntile - 1) / ntile), 128, smem, st>>>(out, in, links, g.nbr, g.V, nb, ld, nrhs, ntile,
                                                                  tmem_cols, err);
  WCMG_LAUNCH_CHECK();
}

size_t coarse_mma4_smem(int nb, int ntile, int mm, int stages) {
  const size_t kg = nb / 4;
  const size_t a_alloc = (kg * nb * 16 + (size_t)(mm > nb ? mm - nb : 0) * 16 + 1023) / 1024 * 1024;
  const size_t b_alloc = (kg * 2 * ntile * 16 + 1023) / 1024 * 1024;
  return (size_t)stages * (a_alloc + b_alloc);
}

size_t coarse_mma4_scratch_bytes(int Vc, int nb, int nrhs) {
  // B operands of every site for any rhs tile of at most 64: Vc x tiles x 2 N x nb x 4 bytes
  return (size_t)Vc * nb * 8 * (size_t)(nrhs + 63);
}

void launch_links_to_mma(bf16c* dst, const bf16c* src, int Vc, int nb, cudaStream_t st) {
  const long long total = (long long)Vc * 9 * (nb / 4) * nb;
  k_links_to_mma<<<nblk(total, 256), 256, 0, st>>>(reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src),
                                                   Vc, nb, links_ld(nb));
  WCMG_LAUNCH_CHECK();
}

static void coarse_apply_mma4(float2* out, const float2* in, const bf16c* lmma, const LevelGeom& g, int nb, int nrhs,
                              const CoarseTile& t, void* scratch, size_t scratch_bytes, int* err, cudaStream_t st) {
  const int ntiles = (nrhs + t.ntile - 1) / t.ntile;
  const long long groups = (long long)g.V * ntiles * (nb / 4) * 2 * t.ntile;
  if ((size_t)groups * 16 > scratch_bytes) throw Error(-1, "coarse apply: tensor-core scratch too small");
  uint4* bp = reinterpret_cast<uint4*>(scratch);
  k_mma_bprep<<<nblk(groups, 256), 256, 0, st>>>(bp, in, g.V, nb, nrhs, t.ntile, ntiles);
  WCMG_LAUNCH_CHECK();
  const size_t smem = coarse_mma4_smem(nb, t.ntile, t.threads, t.stages);
  auto kern = t.threads == 64 ? k_coarse_apply_mma4<64> : k_coarse_apply_mma4<128>;
  WCMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // TMEM: two accumulators of 2 N FP32 columns, each 64 columns wide when 2 N <= 64 (the
  // allocation, a power of two, is then 128 of the SM's 512 columns) else 128.  CTAs per
  // SM as shared memory allows and as many as the TMEM holds.
  // t.parts = 1: one accumulator (the MMAs of the next item wait for the epilogue), half
  // the TMEM, so more CTAs fit an SM
  const int acc_cols = 2 * t.ntile <= 64 ? 64 : 128, nacc = t.parts == 1 ? 1 : 2;
  const int per_sm = std::max(1, std::min(blocks_per_sm((const void*)kern, 192, smem), 512 / (nacc * acc_cols)));
  const long long items = (long long)g.V * ntiles;
  const int grid = (int)std::min<long long>(items, (long long)sm_count() * per_sm);
  kern<<<grid, 192, smem, st>>>(out, reinterpret_cast<const uint4*>(lmma), bp, g.nbr, g.V, nb, nrhs, t.ntile, ntiles,
                                t.stages, acc_cols, nacc, err);
  WCMG_LAUNCH_CHECK();
}

// The fixed launch rule (used unless a tile is given):
//  - BF16 links, full stencil, >= 8 rhs, nbasis <= 64: tensor cores, N tile = rhs rounded to 16 (<= 64);
//  - one rhs, full stencil: the one-rhs kernel, 512 threads, a site split in up to 4
//    CTAs while there are fewer than 2 CTAs per SM;
//  - otherwise the rhs-tile kernel, 4 rhs per CTA (FP64 or <= 4 rhs) else 8, rows split
//    until about 6 CTAs per SM.
CoarseTile coarse_default_tile(int nb, int nrhs, int mode, int Vc, int link_kind) {
  CoarseTile t;
  if (link_kind == 2 && mode == ST_FULL && nrhs >= 8 && nb <= 64) {
    t.kind = 2;
    t.ntile = std::min(64, (nrhs + 15) / 16 * 16);
    return t;
  }
  if (nrhs == 1 && mode == ST_FULL) {
    t.kind = 0;
    t.rr = 1;
    t.parts = 1;
    while (t.parts < 4 && (long long)Vc * t.parts < 2LL * 152) t.parts *= 2;
    t.threads = 512;
    return t;
  }
  t.kind = 1;
  t.rr = nrhs == 1 ? 1 : (nrhs <= 4 || link_kind == 0) ? 4 : 8;
  t.parts = 0;  // automatic
  return t;
}

template <typename L> struct LinkKind;
template <> struct LinkKind<double2> { static constexpr int v = 0; };
template <> struct LinkKind<float2> { static constexpr int v = 1; };
template <> struct LinkKind<bf16c> { static constexpr int v = 2; };
template <> struct LinkKind<f16c> { static constexpr int v = 3; };

bool coarse_tile_valid(const CoarseTile& t, int nb, int nrhs, int mode, int link_kind) {
  switch (t.kind) {
    case 0: {
      // stages: rows in flight per warp (0 or 1: one, 2: two; two only while a row is <= 8 chunks per lane)
      const int vec = link_kind == 0 ? 1 : link_kind == 1 ? 2 : 4;
      const int nk = (links_ld(nb) + 32 * vec - 1) / (32 * vec);
      return nrhs == 1 && mode == ST_FULL && t.parts >= 1 && t.parts <= nb && t.threads >= 64 && t.threads <= 512 &&
             t.threads % 32 == 0 && t.stages >= 0 && t.stages <= 2 && (t.stages < 2 || nk <= 8);
    }
    case 1:
      return (t.rr == 1 || t.rr == 4 || t.rr == 8) && t.parts >= 0 && t.parts <= nb;
    case 2:
      return link_kind == 2 && mode == ST_FULL && nb <= 64 &&
             (t.ntile == 16 || t.ntile == 32 || t.ntile == 48 || t.ntile == 64);
    case 4:
      return link_kind == 2 && mode == ST_FULL && nrhs >= 2 && nb % 8 == 0 && nb <= 64 &&
             (t.parts == 0 || t.parts == 1 || t.parts == 2) &&
             (t.threads == 64 || t.threads == 128) && t.threads >= nb && t.ntile % 8 == 0 && t.ntile >= 8 &&
             t.ntile <= 64 && t.stages >= 2 && t.stages <= MMA4_MAX_STAGES &&
             coarse_mma4_smem(nb, t.ntile, t.threads, t.stages) <= 220 * 1024;
    case 5: {
      // one CTA per site (parts 1); stages: rows in flight per warp (0 or 1: one, 2: two while
      // a row is <= 4 chunks per lane); shared memory within the default 48 KB
      const int vec = link_kind == 0 ? 1 : link_kind == 1 ? 2 : 4;
      const int nk = (links5_ld(nb) + 32 * vec - 1) / (32 * vec);
      const int vb = link_kind == 0 ? 16 : 8;
      const bool vbk = nb % vec == 0 && nb / vec <= t.threads;
      const size_t smem = (size_t)(links5_ld(nb) + 5 * nb + (size_t)(vbk ? t.threads / (nb / vec) : 4) * nb) * vb;
      return nrhs == 1 && mode == ST_FULL && t.parts == 1 && t.threads >= 64 && t.threads <= 512 &&
             t.threads % 32 == 0 && t.stages >= 0 && t.stages <= 2 && (t.stages < 2 || nk <= 4) && nk <= 12 &&
             smem <= 48 * 1024;
    }
    case 3: {
      const int lb = link_kind == 0 ? 16 : link_kind == 1 ? 8 : 4;
      const int vb = link_kind == 0 ? 16 : 8;
      return nrhs == 1 && mode == ST_FULL && (t.threads == 128 || t.threads == 256 || t.threads == 512) &&
             4 * t.threads >= links_ld(nb) &&
             t.parts >= 1 && t.parts <= nb && t.stages >= 2 && t.stages <= STREAM_MAX_STAGES &&
             coarse_stream_smem(nb, t.parts, t.stages, vb, lb) <= 200 * 1024;
    }
    default:
      return false;
  }
}

template <typename R, typename L>
void launch_coarse_apply(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb, int nrhs,
                         int mode, int hopdir, cudaStream_t st, int* err, const CoarseTile* tile, const bf16c* lmma,
                         void* scratch, size_t scratch_bytes, const L* links5) {
  constexpr int lk = LinkKind<L>::v;
  CoarseTile t = coarse_default_tile(nb, nrhs, mode, g.V, lk);
  if (tile && tile->kind >= 0) {
    if (!coarse_tile_valid(*tile, nb, nrhs, mode, lk)) throw Error(-1, "coarse apply: invalid launch tile");
    t = *tile;
  }
  if (t.kind == 2 && !err) t = coarse_default_tile(nb, nrhs, mode, g.V, lk == 2 ? 1 : lk);
  if (t.kind == 2) {
    if constexpr (std::is_same<L, bf16c>::value) {
      coarse_apply_mma<L>((float2*)out, (const float2*)in, links, g, nb, nrhs, t.ntile, err, st);
      return;
    }
    throw Error(-1, "coarse apply: tensor-core tile needs BF16 links");
  }
  if (t.kind == 3 && !err) t = coarse_default_tile(nb, nrhs, mode, g.V, lk);
  if (t.kind == 4 && (!err || !lmma || !scratch)) t = coarse_default_tile(nb, nrhs, mode, g.V, lk);
  if (t.kind == 4) {
    if constexpr (std::is_same<L, bf16c>::value) {
      coarse_apply_mma4((float2*)out, (const float2*)in, lmma, g, nb, nrhs, t, scratch, scratch_bytes, err, st);
      return;
    }
    throw Error(-1, "coarse apply: tensor-core tile needs BF16 links");
  }
  if (t.kind == 5 && !links5) t = coarse_default_tile(nb, nrhs, mode, g.V, lk);
  if (t.kind == 5) {
    coarse_apply5<R, L>(out, in, links5, g, nb, t.threads, t.stages == 2 ? 2 : 1, st);
    return;
  }
  if (t.kind == 0) {
    coarse_apply1<R, L>(out, in, links, g, nb, t.parts, t.threads, t.stages == 2 ? 2 : 1, st);
    return;
  }
  if (t.kind == 3) {
    coarse_apply1_stream<R, L>(out, in, links, g, nb, t.threads, t.parts, t.stages, err, st);
    return;
  }
  // masked applies of the Galerkin construction with several fields: one GEMM per site
  // (FP64 / FP32 link storage, nbasis <= 64, shared memory within the SM's 227 KB)
  if constexpr (std::is_same<L, double2>::value || std::is_same<L, float2>::value) {
    if ((mode == ST_BLOCK_INTERIOR || mode == ST_FACE_HOP) && nrhs >= 2 && nb <= 64 &&
        coarse_masked_gemm_smem(nb, nrhs, (int)sizeof(cplx<R>)) <= 200 * 1024 && (!tile || tile->kind < 0)) {
      coarse_masked_gemm<R, L>(out, in, links, g, nb, nrhs, mode, hopdir, st);
      return;
    }
  }
  if (t.rr == 1) coarse_apply_rr<R, L, 1>(out, in, links, g, nb, nrhs, mode, hopdir, t.parts, st);
  else if (t.rr == 4) coarse_apply_rr<R, L, 4>(out, in, links, g, nb, nrhs, mode, hopdir, t.parts, st);
  else coarse_apply_rr<R, L, 8>(out, in, links, g, nb, nrhs, mode, hopdir, t.parts, st);
}

// ---------------- link packing / assembly ----------------
template <typename L>
__global__ void k_pack_links(L* __restrict__ links, const double2* __restrict__ ext, const int* __restrict__ perm,
                             int Vc, int nb, int ld) {
  const int s = blockIdx.x;
  const int lex = perm[s];
  for (int idx = threadIdx.x; idx < nb * ld; idx += blockDim.x) {
    const int a = idx / ld, k = idx % ld;
    double2 v = make_double2(0, 0);
    if (k < 9 * nb) {
      const int d = k / nb, b = k % nb;
      v = ext[(((long long)d * Vc + lex) * nb + a) * nb + b];
    }
    links[(long long)s * nb * ld + idx] = link_store<L>(v);
  }
}

template <typename L>
__global__ void k_unpack_links(double2* __restrict__ ext, const L* __restrict__ links, const int* __restrict__ perm,
                               int Vc, int nb, int ld) {
  const int s = blockIdx.x;
  const int lex = perm[s];
  for (int idx = threadIdx.x; idx < 9 * nb * nb; idx += blockDim.x) {
    const int d = idx / (nb * nb), a = (idx / nb) % nb, b = idx % nb;
    ext[(((long long)d * Vc + lex) * nb + a) * nb + b] = link_to_c64<L>(links[((long long)s * nb + a) * ld + d * nb + b]);
  }
}

template <typename R, typename L>
__global__ void k_scatter_links(L* __restrict__ links, const cplx<R>* __restrict__ res, int Vc, int nb, int ld, int d,
                                int b0, int ncols) {
  const int x = blockIdx.x;
  for (int idx = threadIdx.x; idx < ncols * nb; idx += blockDim.x) {
    const int j = idx / nb, a = idx % nb;
    links[((long long)x * nb + a) * ld + d * nb + b0 + j] = link_store<L>(to_c64(res[((long long)j * Vc + x) * nb + a]));
  }
}

template <typename Lin, typename Lout>
__global__ void k_convert_links(Lout* __restrict__ out, const Lin* __restrict__ in, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) out[i] = link_store<Lout>(link_to_c64<Lin>(in[i]));
}

template <typename R>
__global__ void k_pack_coarse(cplx<R>* __restrict__ out, const double2* __restrict__ ext, const int* __restrict__ perm,
                              int V, int nc) {
  const int s = blockIdx.x, r = blockIdx.y;
  const int lex = perm[s];
  for (int c = threadIdx.x; c < nc; c += blockDim.x)
    out[((long long)r * V + s) * nc + c] = from_c64<R>(ext[((long long)r * V + lex) * nc + c]);
}
template <typename R>
__global__ void k_unpack_coarse(double2* __restrict__ ext, const cplx<R>* __restrict__ in, const int* __restrict__ perm,
                                int V, int nc) {
  const int s = blockIdx.x, r = blockIdx.y;
  const int lex = perm[s];
  for (int c = threadIdx.x; c < nc; c += blockDim.x)
    ext[((long long)r * V + lex) * nc + c] = to_c64(in[((long long)r * V + s) * nc + c]);
}

template <typename L>
void launch_pack_links(L* links, const double2* ext, const int* perm, int Vc, int nb, cudaStream_t st) {
  k_pack_links<L><<<Vc, 256, 0, st>>>(links, ext, perm, Vc, nb, links_ld(nb));
  WCMG_LAUNCH_CHECK();
}
template <typename L>
void launch_unpack_links(double2* ext, const L* links, const int* perm, int Vc, int nb, cudaStream_t st) {
  k_unpack_links<L><<<Vc, 256, 0, st>>>(ext, links, perm, Vc, nb, links_ld(nb));
  WCMG_LAUNCH_CHECK();
}
template <typename R, typename L>
void launch_scatter_links(L* links, const cplx<R>* res, int Vc, int nb, int d, int b0, int ncols, cudaStream_t st) {
  k_scatter_links<R, L><<<Vc, 256, 0, st>>>(links, res, Vc, nb, links_ld(nb), d, b0, ncols);
  WCMG_LAUNCH_CHECK();
}
template <typename Lin, typename Lout>
void launch_convert_links(Lout* out, const Lin* in, long long n, cudaStream_t st) {
  k_convert_links<Lin, Lout><<<nblk(n, 256), 256, 0, st>>>(out, in, n);
  WCMG_LAUNCH_CHECK();
}
template <typename R>
void launch_pack_coarse(cplx<R>* out, const double2* ext, const int* perm, int V, int nc, int nrhs, cudaStream_t st) {
  k_pack_coarse<R><<<dim3(V, nrhs), 64, 0, st>>>(out, ext, perm, V, nc);
  WCMG_LAUNCH_CHECK();
}
template <typename R>
void launch_unpack_coarse(double2* ext, const cplx<R>* in, const int* perm, int V, int nc, int nrhs, cudaStream_t st) {
  k_unpack_coarse<R><<<dim3(V, nrhs), 64, 0, st>>>(ext, in, perm, V, nc);
  WCMG_LAUNCH_CHECK();
}

template void launch_coarse_apply<double, double2>(double2*, const double2*, const double2*, const LevelGeom&, int,
                                                   int, int, int, cudaStream_t, int*, const CoarseTile*,
                                                   const bf16c*, void*, size_t, const double2*);
template void launch_coarse_apply<float, float2>(float2*, const float2*, const float2*, const LevelGeom&, int, int,
                                                 int, int, cudaStream_t, int*, const CoarseTile*,
                                                   const bf16c*, void*, size_t, const float2*);
template void launch_coarse_apply<float, bf16c>(float2*, const float2*, const bf16c*, const LevelGeom&, int, int, int,
                                                int, cudaStream_t, int*, const CoarseTile*,
                                                const bf16c*, void*, size_t, const bf16c*);
template void launch_coarse_apply<float, f16c>(float2*, const float2*, const f16c*, const LevelGeom&, int, int, int,
                                               int, cudaStream_t, int*, const CoarseTile*,
                                                const bf16c*, void*, size_t, const f16c*);
#define WCMG_INST_L(L)                                                                                   \
  template void launch_links_to_5<L>(L*, const L*, int, int, cudaStream_t);                             \
  template void launch_pack_links<L>(L*, const double2*, const int*, int, int, cudaStream_t);           \
  template void launch_unpack_links<L>(double2*, const L*, const int*, int, int, cudaStream_t);
WCMG_INST_L(double2)
WCMG_INST_L(float2)
WCMG_INST_L(bf16c)
WCMG_INST_L(f16c)
#undef WCMG_INST_L
template void launch_scatter_links<double, double2>(double2*, const double2*, int, int, int, int, int, cudaStream_t);
template void launch_scatter_links<float, float2>(float2*, const float2*, int, int, int, int, int, cudaStream_t);
template void launch_convert_links<float2, bf16c>(bf16c*, const float2*, long long, cudaStream_t);
template void launch_convert_links<float2, f16c>(f16c*, const float2*, long long, cudaStream_t);
template void launch_convert_links<double2, float2>(float2*, const double2*, long long, cudaStream_t);
template void launch_convert_links<double2, bf16c>(bf16c*, const double2*, long long, cudaStream_t);
template void launch_convert_links<double2, f16c>(f16c*, const double2*, long long, cudaStream_t);
#define WCMG_INST(R)                                                                                     \
  template void launch_pack_coarse<R>(cplx<R>*, const double2*, const int*, int, int, int, cudaStream_t); \
  template void launch_unpack_coarse<R>(double2*, const cplx<R>*, const int*, int, int, int, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST

}  // namespace wcmg
