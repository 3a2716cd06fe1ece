// Fine-level kernels: layout packing, gauge field, clover term (K0) and the
// Wilson-clover Dslash (K1).
//
// Operator (Sec. 2.1: multigrid runs on the Wilson-clover D itself; Sec. 2.2:
// chiral gamma basis so that gamma5 = diag(1, 1, -1, -1)):
//   D psi(x) = C(x) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                      + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu) ]
// with gamma_mu = [[0, B_mu], [B_mu^dag, 0]], B_k = -i sigma_k (k = x, y, z),
// B_t = 1.  The (1 -+ gamma_mu) projectors are applied as 2-spin half spinors:
//   forward : h = psi_u - B psi_l,  upper += U h,      lower += -B^dag (U h)
//   backward: h = psi_u + B psi_l,  upper += U^dag h,  lower += +B^dag (U^dag h)
// C(x) = (4 + m0) + (c_sw/2) sum_{mu<nu} sigma_{mu nu} (x) i Fhat_{mu nu}(x) is
// block diagonal in chirality (two Hermitian 6x6 blocks), stored compactly:
// per chirality 3 pairs of real diagonal entries and 15 complex upper entries.
//
// Internal layouts (storage order of sites, see LevelGeom):
//   spinor : [12][V] complex   (component c = 3 * spin + colour)
//   gauge  : [4][9][V] complex (entry (mu, 3 a + b) = U_mu(x)[a][b])
//   clover : [36][V] complex   (chirality s uses entries 18 s .. 18 s + 17)
#include "kernels.h"

namespace wcmg {

// ---------------- packing ----------------
template <typename R>
__global__ void k_pack_fine(cplx<R>* __restrict__ out, const double2* __restrict__ ext, const int* __restrict__ perm,
                            int V, int nrhs) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (s >= V) return;
  const double2* e = ext + ((long long)r * V + perm[s]) * 12;
  cplx<R>* o = out + (long long)r * 12 * V;
#pragma unroll
  for (int c = 0; c < 12; ++c) o[(long long)c * V + s] = from_c64<R>(e[c]);
}

template <typename R>
__global__ void k_unpack_fine(double2* __restrict__ ext, const cplx<R>* __restrict__ in, const int* __restrict__ perm,
                              int V, int nrhs) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (s >= V) return;
  double2* e = ext + ((long long)r * V + perm[s]) * 12;
  const cplx<R>* i = in + (long long)r * 12 * V;
#pragma unroll
  for (int c = 0; c < 12; ++c) e[c] = to_c64(i[(long long)c * V + s]);
}

template <typename R>
__global__ void k_pack_gauge(cplx<R>* __restrict__ out, const double2* __restrict__ ext, const int* __restrict__ perm,
                             int V) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  int mu = blockIdx.y;
  if (s >= V) return;
  const double2* e = ext + ((long long)mu * V + perm[s]) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) out[((long long)mu * 9 + k) * V + s] = from_c64<R>(e[k]);
}

template <typename R>
void launch_pack_fine(cplx<R>* out, const double2* ext, const int* perm, int V, int nrhs, cudaStream_t st) {
  k_pack_fine<R><<<dim3(nblk(V, 128), nrhs), 128, 0, st>>>(out, ext, perm, V, nrhs);
  WCMG_LAUNCH_CHECK();
}
template <typename R>
void launch_unpack_fine(double2* ext, const cplx<R>* in, const int* perm, int V, int nrhs, cudaStream_t st) {
  k_unpack_fine<R><<<dim3(nblk(V, 128), nrhs), 128, 0, st>>>(ext, in, perm, V, nrhs);
  WCMG_LAUNCH_CHECK();
}
template <typename R>
void launch_pack_gauge(cplx<R>* out, const double2* ext, const int* perm, int V, cudaStream_t st) {
  k_pack_gauge<R><<<dim3(nblk(V, 128), 4), 128, 0, st>>>(out, ext, perm, V);
  WCMG_LAUNCH_CHECK();
}

// ---------------- clover term (K0, FP64, once per gauge field) ----------------
struct Su3 { double2 m[9]; };

__device__ __forceinline__ Su3 load_u(const double2* __restrict__ g, int V, int mu, int s) {
  Su3 u;
#pragma unroll
  for (int k = 0; k < 9; ++k) u.m[k] = g[((long long)mu * 9 + k) * V + s];
  return u;
}
__device__ __forceinline__ Su3 dag(const Su3& a) {
  Su3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.m[3 * i + j] = conjg(a.m[3 * j + i]);
  return r;
}
__device__ __forceinline__ Su3 mm(const Su3& a, const Su3& b) {
  Su3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 acc = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc, a.m[3 * i + k], b.m[3 * k + j]);
      r.m[3 * i + j] = acc;
    }
  return r;
}

// S[plane][chirality][2x2]: the chiral blocks of sigma_{mu nu} = i gamma_mu gamma_nu
// (upper: i B_mu B_nu^dag, lower: i B_mu^dag B_nu), planes in the order
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3).
struct CloverSigma { double2 S[6][2][4]; };

__global__ void k_clover_build(double2* __restrict__ clov, const double2* __restrict__ g, const int* __restrict__ nbr,
                               int V, double diag, double half_csw, CloverSigma sig) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double2 C[2][6][6];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 6; ++j) C[h][i][j] = make_double2(i == j ? diag : 0.0, 0.0);
  int plane = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
      const int xpm = nbr[(2 * mu) * V + s], xmm = nbr[(2 * mu + 1) * V + s];
      const int xpn = nbr[(2 * nu) * V + s], xmn = nbr[(2 * nu + 1) * V + s];
      const int xmm_pn = nbr[(2 * nu) * V + xmm];      // x - mu + nu
      const int xmm_mn = nbr[(2 * nu + 1) * V + xmm];  // x - mu - nu
      const int xpm_mn = nbr[(2 * nu + 1) * V + xpm];  // x + mu - nu
      Su3 Umx = load_u(g, V, mu, s), Unx = load_u(g, V, nu, s);
      Su3 Um_mm = load_u(g, V, mu, xmm), Un_mn = load_u(g, V, nu, xmn);
      // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      Su3 Q = mm(mm(Umx, load_u(g, V, nu, xpm)), mm(dag(load_u(g, V, mu, xpn)), dag(Unx)));
      // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
      Su3 L = mm(mm(Unx, dag(load_u(g, V, mu, xmm_pn))), mm(dag(load_u(g, V, nu, xmm)), Um_mm));
#pragma unroll
      for (int k = 0; k < 9; ++k) Q.m[k] += L.m[k];
      // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
      L = mm(mm(dag(Um_mm), dag(load_u(g, V, nu, xmm_mn))), mm(load_u(g, V, mu, xmm_mn), Un_mn));
#pragma unroll
      for (int k = 0; k < 9; ++k) Q.m[k] += L.m[k];
      // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
      L = mm(mm(dag(Un_mn), load_u(g, V, mu, xmn)), mm(load_u(g, V, nu, xpm_mn), dag(Umx)));
#pragma unroll
      for (int k = 0; k < 9; ++k) Q.m[k] += L.m[k];
      // i Fhat = i (Q - Q^dag) / 8  (Hermitian)
      double2 iF[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) iF[3 * a + b] = mul_i(0.125 * (Q.m[3 * a + b] - conjg(Q.m[3 * b + a])));
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const double2 sp = half_csw * sig.S[plane][h][2 * p + q];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b) cmac(C[h][3 * p + a][3 * q + b], sp, iF[3 * a + b]);
          }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      clov[(long long)(18 * h + k) * V + s] = make_double2(C[h][2 * k][2 * k].x, C[h][2 * k + 1][2 * k + 1].x);
    int o = 3;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) clov[(long long)(18 * h + o++) * V + s] = C[h][i][j];
  }
}

__global__ void k_clover_expand(double2* __restrict__ ext, const double2* __restrict__ clov,
                                const int* __restrict__ perm, int V) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double2* e = ext + (long long)perm[s] * 144;
  for (int k = 0; k < 144; ++k) e[k] = make_double2(0, 0);
  for (int h = 0; h < 2; ++h) {
    for (int k = 0; k < 3; ++k) {
      double2 d = clov[(long long)(18 * h + k) * V + s];
      e[(6 * h + 2 * k) * 12 + 6 * h + 2 * k] = make_double2(d.x, 0);
      e[(6 * h + 2 * k + 1) * 12 + 6 * h + 2 * k + 1] = make_double2(d.y, 0);
    }
    int o = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) {
        double2 c = clov[(long long)(18 * h + o++) * V + s];
        e[(6 * h + i) * 12 + 6 * h + j] = c;
        e[(6 * h + j) * 12 + 6 * h + i] = conjg(c);
      }
  }
}

// Inverse of k_clover_expand for caller-given site blocks (wcmg_set_clover_raw).
// The packed layout keeps the two chiral 6x6 blocks only, with the diagonal real
// and the upper triangle: a block that is not Hermitian and block diagonal could
// not be represented, so such a site raises *bad instead of being truncated.
__global__ void k_clover_pack(double2* __restrict__ clov, const double2* __restrict__ ext,
                              const int* __restrict__ perm, int V, double tol, int* __restrict__ bad) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const double2* e = ext + (long long)perm[s] * 144;
  double scale = 0.0, dev = 0.0;
  bool finite = true;
  for (int i = 0; i < 12; ++i)
    for (int j = 0; j < 12; ++j) {
      const double2 a = e[i * 12 + j];
      finite &= isfinite(a.x) && isfinite(a.y);
      const double m = fabs(a.x) + fabs(a.y);
      scale = fmax(scale, m);
      if ((i < 6) != (j < 6)) {
        dev = fmax(dev, m);  // couples the two chiralities
      } else if (j >= i) {
        const double2 b = e[j * 12 + i];
        dev = fmax(dev, fabs(a.x - b.x) + fabs(a.y + b.y));  // a != conj(b)
      }
    }
  if (!finite || dev > tol * scale) atomicOr(bad, 1);
  for (int h = 0; h < 2; ++h) {
    for (int k = 0; k < 3; ++k)
      clov[(long long)(18 * h + k) * V + s] =
          make_double2(e[(6 * h + 2 * k) * 12 + 6 * h + 2 * k].x, e[(6 * h + 2 * k + 1) * 12 + 6 * h + 2 * k + 1].x);
    int o = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j) clov[(long long)(18 * h + o++) * V + s] = e[(6 * h + i) * 12 + 6 * h + j];
  }
}

static CloverSigma make_sigma() {
  // B_mu as 2x2 complex (row-major)
  double2 B[4][4];
  const double2 z = make_double2(0, 0), one = make_double2(1, 0), mi = make_double2(0, -1);
  // B_x = -i sigma_1 ; B_y = -i sigma_2 ; B_z = -i sigma_3 ; B_t = 1
  double2 Bx[4] = {z, mi, mi, z};
  double2 By[4] = {z, make_double2(-1, 0), one, z};
  double2 Bz[4] = {mi, z, z, make_double2(0, 1)};
  double2 Bt[4] = {one, z, z, one};
  for (int k = 0; k < 4; ++k) { B[0][k] = Bx[k]; B[1][k] = By[k]; B[2][k] = Bz[k]; B[3][k] = Bt[k]; }
  auto mul = [](const double2* a, const double2* b, double2* r, bool dag_a, bool dag_b) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double2 acc = make_double2(0, 0);
        for (int k = 0; k < 2; ++k) {
          double2 x = dag_a ? conjg(a[2 * k + i]) : a[2 * i + k];
          double2 y = dag_b ? conjg(b[2 * j + k]) : b[2 * k + j];
          acc += cmul(x, y);
        }
        r[2 * i + j] = mul_i(acc);
      }
  };
  CloverSigma cs;
  int plane = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++plane) {
      mul(B[mu], B[nu], cs.S[plane][0], false, true);   // i B_mu B_nu^dag
      mul(B[mu], B[nu], cs.S[plane][1], true, false);   // i B_mu^dag B_nu
    }
  return cs;
}

void launch_clover_build(double2* clov, const double2* gauge64, const int* nbr, int V, double m0, double csw,
                         cudaStream_t st) {
  static const CloverSigma sig = make_sigma();
  k_clover_build<<<nblk(V, 64), 64, 0, st>>>(clov, gauge64, nbr, V, 4.0 + m0, 0.5 * csw, sig);
  WCMG_LAUNCH_CHECK();
}
void launch_clover_expand(double2* ext, const double2* clov, const int* perm, int V, cudaStream_t st) {
  k_clover_expand<<<nblk(V, 128), 128, 0, st>>>(ext, clov, perm, V);
  WCMG_LAUNCH_CHECK();
}
void launch_clover_pack(double2* clov, const double2* ext, const int* perm, int V, double tol, int* bad,
                        cudaStream_t st) {
  k_clover_pack<<<nblk(V, 128), 128, 0, st>>>(clov, ext, perm, V, tol, bad);
  WCMG_LAUNCH_CHECK();
}

// ---------------- Dslash (K1) ----------------
// apply B_mu (or B_mu^dag) to a 2-spin x 3-colour half spinor v[2][3]
template <int MU, typename T>
__device__ __forceinline__ void applyB(T (&out)[2][3], const T (&v)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { out[0][c] = mul_mi(v[1][c]); out[1][c] = mul_mi(v[0][c]); }
    if (MU == 1) { out[0][c] = -v[1][c]; out[1][c] = v[0][c]; }
    if (MU == 2) { out[0][c] = mul_mi(v[0][c]); out[1][c] = mul_i(v[1][c]); }
    if (MU == 3) { out[0][c] = v[0][c]; out[1][c] = v[1][c]; }
  }
}
template <int MU, typename T>
__device__ __forceinline__ void applyBdag(T (&out)[2][3], const T (&v)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (MU == 0) { out[0][c] = mul_i(v[1][c]); out[1][c] = mul_i(v[0][c]); }
    if (MU == 1) { out[0][c] = v[1][c]; out[1][c] = -v[0][c]; }
    if (MU == 2) { out[0][c] = mul_i(v[0][c]); out[1][c] = mul_mi(v[1][c]); }
    if (MU == 3) { out[0][c] = v[0][c]; out[1][c] = v[1][c]; }
  }
}

// One hop of the stencil for NR right-hand sides at once: the link (U_mu(x) forward,
// U_mu(x - mu)^dag backward) is loaded once and applied to every rhs's
// projected half spinor.
// The neighbour spinor is read from `in` as component c at in[c * vin + yin] (the
// field itself: vin = V, yin = the neighbour's site; a block staged in shared memory:
// its own stride and local index); the link from U at storage site ls.
template <typename R, int MU, bool FWD, int NR>
__device__ __forceinline__ void hop_at(cplx<R> (&acc)[NR][12], const cplx<R>* __restrict__ in, long long rstride,
                                       int vin, int yin, const cplx<R>* __restrict__ U, int V, int ls) {
  using T = cplx<R>;
  T u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = U[((long long)MU * 9 + k) * V + ls];
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    const cplx<R>* iq = in + q * rstride;
    T pu[2][3], pl[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pu[sp][c] = iq[(long long)(3 * sp + c) * vin + yin];
        pl[sp][c] = iq[(long long)(6 + 3 * sp + c) * vin + yin];
      }
    T Bpl[2][3], h[2][3];
    applyB<MU>(Bpl, pl);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) h[sp][c] = FWD ? pu[sp][c] - Bpl[sp][c] : pu[sp][c] + Bpl[sp][c];
    T w[2][3];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T t = czero<R>();
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (FWD) cmac(t, u[3 * a + b], h[sp][b]);
          else cjmac(t, u[3 * b + a], h[sp][b]);
        }
        w[sp][a] = t;
      }
    T Bw[2][3];
    applyBdag<MU>(Bw, w);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[q][3 * sp + c] += w[sp][c];
        if (FWD) acc[q][6 + 3 * sp + c] -= Bw[sp][c];
        else acc[q][6 + 3 * sp + c] += Bw[sp][c];
      }
  }
}

template <typename R, int MU, bool FWD, int NR>
__device__ __forceinline__ void hop(cplx<R> (&acc)[NR][12], const cplx<R>* __restrict__ in, long long rstride,
                                    const cplx<R>* __restrict__ U, int V, int s, int y) {
  hop_at<R, MU, FWD, NR>(acc, in, rstride, V, y, U, V, FWD ? s : y);  // link U_mu(x) fwd, U_mu(x - mu) bwd
}

// acc_q = C(x) psi_q - acc_q / 2 for the components of chirality half h (NR rhs;
// each clover entry is loaded once); p holds psi_q's six components of half h.
template <typename R, int NR>
__device__ __forceinline__ void clover_half(cplx<R> (&acc)[NR][12], const cplx<R>* __restrict__ clov,
                                            const cplx<R> (&p)[NR][6], int h, int V, int s) {
  using T = cplx<R>;
#pragma unroll
  for (int q = 0; q < NR; ++q)
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[q][6 * h + i] = R(-0.5) * acc[q][6 * h + i];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T d = clov[(long long)(18 * h + k) * V + s];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      acc[q][6 * h + 2 * k] += d.x * p[q][2 * k];
      acc[q][6 * h + 2 * k + 1] += d.y * p[q][2 * k + 1];
    }
  }
  int o = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const T c = clov[(long long)(18 * h + o++) * V + s];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        cmac(acc[q][6 * h + i], c, p[q][j]);
        cjmac(acc[q][6 * h + j], c, p[q][i]);
      }
    }
}

struct BlockInfo { int b[4]; int bvol; };

__device__ __forceinline__ bool on_face(const BlockInfo& bi, int s, int d) {
  int loc = s % bi.bvol;
  int l[4];
  l[0] = loc % bi.b[0]; loc /= bi.b[0];
  l[1] = loc % bi.b[1]; loc /= bi.b[1];
  l[2] = loc % bi.b[2];
  l[3] = loc / bi.b[2];
  const int mu = d >> 1;
  return (d & 1) ? (l[mu] == 0) : (l[mu] == bi.b[mu] - 1);
}

// MR epilogue (DOTS): the CTA also sums <out, in> = sum conj(out) in and <out, out>
// over its sites (FP32/FP64 per thread, FP64 across the CTA) into one partial per
// (rhs, CTA): the minimal-residual step p = D r, alpha = <p, r>/<p, p> then needs
// no extra pass over p and r.
template <typename R, int MODE, bool DOTS, int NR>
__global__ void __launch_bounds__(128, (sizeof(R) == 4 && NR == 1) ? 6 : (sizeof(R) == 4 ? 4 : 1))
    k_dslash(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in, const cplx<R>* __restrict__ U,
             const cplx<R>* __restrict__ clov, const int* __restrict__ nbr, int V, BlockInfo bi, int hopdir, int nrhs,
             double2* __restrict__ pr_part, double* __restrict__ pp_part,
             const unsigned char* __restrict__ colour, int col) {
  using T = cplx<R>;
  // rhs groups fastest in the grid: the CTAs running together cover the same sites
  // for every rhs, so links and clover are fetched from HBM once
  const int ngrp = (nrhs + NR - 1) / NR;
  const int grp = blockIdx.x % ngrp;
  const int r0 = grp * NR;
  const int nq = min(NR, nrhs - r0);  // rhs of this thread (the last group may be short)
  const int s = (blockIdx.x / ngrp) * blockDim.x + threadIdx.x;
  const bool valid = s < V;
  if (!DOTS && !valid) return;
  // single-face mode: sites off the face are never read by the face restriction
  if (MODE == ST_FACE_HOP && !on_face(bi, s, hopdir)) return;
  // SAP residual: only the aggregates of one colour (the other sites are not written)
  if (!DOTS && colour && colour[s / bi.bvol] != col) return;
  const long long rstride = 12LL * V;
  // a short last group re-reads its last rhs (nothing of it is stored)
  const long long off = (long long)r0 * rstride;
  const cplx<R>* inr = in + off;
  const long long rs = nq > 1 ? rstride : 0;
  R dr[NR], di[NR], nn[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) dr[q] = di[q] = nn[q] = 0;
  if (valid) {
    T acc[NR][12];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[q][c] = czero<R>();
    auto use = [&](int d) -> bool {
      if (MODE == ST_FULL) return true;
      if (MODE == ST_BLOCK_INTERIOR) return !on_face(bi, s, d);
      return d == hopdir && on_face(bi, s, d);
    };
#define WCMG_HOP(MU)                                                                             \
  if (use(2 * MU)) hop<R, MU, true, NR>(acc, inr, rs, U, V, s, nbr[(2 * MU) * V + s]);            \
  if (use(2 * MU + 1)) hop<R, MU, false, NR>(acc, inr, rs, U, V, s, nbr[(2 * MU + 1) * V + s]);
    WCMG_HOP(0)
    WCMG_HOP(1)
    WCMG_HOP(2)
    WCMG_HOP(3)
#undef WCMG_HOP
    // epilogue per chirality half: clover term, store, MR reductions
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (MODE != ST_FACE_HOP) {
        T p[NR][6];
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
          for (int i = 0; i < 6; ++i) p[q][i] = inr[q * rs + (long long)(6 * h + i) * V + s];
        clover_half<R, NR>(acc, clov, p, h, V, s);
        if (DOTS) {
#pragma unroll
          for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int i = 0; i < 6; ++i) {
              const T o = acc[q][6 * h + i];
              dr[q] += o.x * p[q][i].x + o.y * p[q][i].y;
              di[q] += o.x * p[q][i].y - o.y * p[q][i].x;
              nn[q] += o.x * o.x + o.y * o.y;
            }
        }
      } else {
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
          for (int i = 0; i < 6; ++i) acc[q][6 * h + i] = R(-0.5) * acc[q][6 * h + i];
      }
#pragma unroll
      for (int q = 0; q < NR; ++q)
        if (q < nq) {
          cplx<R>* oq = out + off + q * rstride;
#pragma unroll
          for (int i = 0; i < 6; ++i) oq[(long long)(6 * h + i) * V + s] = acc[q][6 * h + i];
        }
    }
  }
  if (DOTS) {
    __shared__ double scratch[(128 / 32) * 3 * NR];
    __shared__ double red[3 * NR];
    R v[3 * NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      v[3 * q] = dr[q];
      v[3 * q + 1] = di[q];
      v[3 * q + 2] = nn[q];
    }
    block_sum_mixed<R, 3 * NR>(v, scratch, red);
    if (threadIdx.x < nq) {
      const int q = threadIdx.x;
      const int nsb = gridDim.x / ngrp, sb = blockIdx.x / ngrp;
      pr_part[(long long)(r0 + q) * nsb + sb] = make_double2(red[3 * q], red[3 * q + 1]);
      pp_part[(long long)(r0 + q) * nsb + sb] = red[3 * q + 2];
    }
  }
}

// rhs per thread: 2 for FP32 with several rhs, else 1
template <typename R>
static int dslash_nr(int nrhs) { return (sizeof(R) == 4 && nrhs > 1) ? 2 : 1; }

template <typename R>
void launch_dslash(cplx<R>* out, const cplx<R>* in, const cplx<R>* gauge, const cplx<R>* clov, const LevelGeom& g,
                   int nrhs, int mode, int hopdir, cudaStream_t st, const unsigned char* colour, int col) {
  BlockInfo bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const int nr = dslash_nr<R>(nrhs);
  const dim3 grid((unsigned)(nblk(g.V, 128) * (long long)((nrhs + nr - 1) / nr)));
#define WCMG_DS(MODE, NR) \
  k_dslash<R, MODE, false, NR><<<grid, 128, 0, st>>>(out, in, gauge, clov, g.nbr, g.V, bi, hopdir, nrhs, nullptr, \
                                                     nullptr, colour, col)
  if constexpr (sizeof(R) == 4) {
    if (nr == 2) {
      if (mode == ST_FULL) WCMG_DS(ST_FULL, 2);
      else if (mode == ST_BLOCK_INTERIOR) WCMG_DS(ST_BLOCK_INTERIOR, 2);
      else WCMG_DS(ST_FACE_HOP, 2);
      WCMG_LAUNCH_CHECK();
      return;
    }
  }
  {
    if (mode == ST_FULL) WCMG_DS(ST_FULL, 1);
    else if (mode == ST_BLOCK_INTERIOR) WCMG_DS(ST_BLOCK_INTERIOR, 1);
    else WCMG_DS(ST_FACE_HOP, 1);
  }
#undef WCMG_DS
  WCMG_LAUNCH_CHECK();
}

// ---- SAP colour pass on the fine level (Sec. 4 smoother) ----
// One CTA per aggregate of the pass's colour (blocks[blockIdx.x]), one thread per
// site of it, one rhs per grid row.  The block's residual r = b - D x (b where x = 0)
// stays in shared memory ([12][T], component-major like the field) for all `steps`
// minimal-residual steps of the block-local operator D_B (D without the hops that
// leave the aggregate): p = D_B r from the neighbours' r in shared memory and the
// site's links and clover (HBM once, then L1/L2), alpha_B = <p, r>_B / <p, p>_B summed
// over the block (FP64 across warps), e += alpha_B r, r -= alpha_B p.  x += e at the
// end; only the CTA's own sites are written, so blocks of one colour run concurrently.
constexpr int SAP_FINE_T = 256;
template <typename R>
__global__ void __launch_bounds__(SAP_FINE_T, sizeof(R) == 4 ? 2 : 1)
    k_sap_fine(cplx<R>* __restrict__ x, const cplx<R>* __restrict__ b, const cplx<R>* __restrict__ Dx,
               const cplx<R>* __restrict__ U, const cplx<R>* __restrict__ clov, int V, BlockInfo bi,
               const int* __restrict__ blocks, int steps) {
  using T = cplx<R>;
  extern __shared__ __align__(16) unsigned char sap_smem[];
  T* rs = reinterpret_cast<T*>(sap_smem);
  const int NT = blockDim.x;
  const int i = threadIdx.x;
  const bool valid = i < bi.bvol;
  const int s = blocks[blockIdx.x] * bi.bvol + i;
  const long long off = (long long)blockIdx.y * 12 * V;
  int l[4], st[4];
  {
    int loc = valid ? i : 0;
    st[0] = 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      l[k] = loc % bi.b[k];
      loc /= bi.b[k];
      if (k < 3) st[k + 1] = st[k] * bi.b[k];
    }
  }
  T r[12], e[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    T v = czero<R>();
    if (valid) {
      const long long o = off + (long long)c * V + s;
      v = Dx ? b[o] - Dx[o] : b[o];
    }
    r[c] = v;
    e[c] = czero<R>();
    rs[c * NT + i] = v;
  }
  __syncthreads();
  __shared__ double scratch[(SAP_FINE_T / 32) * 3], red[3];
  for (int k = 0; k < steps; ++k) {
    T acc[1][12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[0][c] = czero<R>();
    R v3[3] = {R(0), R(0), R(0)};
    if (valid) {
#define WCMG_SAP_HOP(MU)                                                                                   \
  if (l[MU] < bi.b[MU] - 1) hop_at<R, MU, true, 1>(acc, rs, 0, NT, i + st[MU], U, V, s);                  \
  if (l[MU] > 0) hop_at<R, MU, false, 1>(acc, rs, 0, NT, i - st[MU], U, V, s - st[MU]);
      WCMG_SAP_HOP(0)
      WCMG_SAP_HOP(1)
      WCMG_SAP_HOP(2)
      WCMG_SAP_HOP(3)
#undef WCMG_SAP_HOP
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        T p[1][6];
#pragma unroll
        for (int j = 0; j < 6; ++j) p[0][j] = r[6 * h + j];
        clover_half<R, 1>(acc, clov, p, h, V, s);
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const T o = acc[0][c];
        v3[0] += o.x * r[c].x + o.y * r[c].y;
        v3[1] += o.x * r[c].y - o.y * r[c].x;
        v3[2] += o.x * o.x + o.y * o.y;
      }
    }
    block_sum_mixed<R, 3>(v3, scratch, red);  // every thread's reads of rs are done here
    const double pp = red[2];
    const T a = pp != 0.0 ? cmk((R)(red[0] / pp), (R)(red[1] / pp)) : czero<R>();
    if (valid) {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cmac(e[c], a, r[c]);
        r[c] = r[c] - cmul(a, acc[0][c]);
        rs[c * NT + i] = r[c];
      }
    }
    __syncthreads();
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const long long o = off + (long long)c * V + s;
      x[o] = x[o] + e[c];
    }
  }
}

int sap_fine_threads(int bvol) {
  if (bvol < 1 || bvol > SAP_FINE_T) return 0;
  return (bvol + 31) / 32 * 32;
}

template <typename R>
void launch_sap_fine(cplx<R>* x, const cplx<R>* b, const cplx<R>* Dx, const cplx<R>* gauge, const cplx<R>* clov,
                     const LevelGeom& g, const int* blocks, int nblocks, int steps, int nrhs, cudaStream_t st) {
  const int nt = sap_fine_threads(g.bvol);
  if (!nt) throw Error(-1, "fused SAP pass needs aggregates of at most 256 sites");
  if (nblocks <= 0) return;
  BlockInfo bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const size_t smem = (size_t)12 * nt * sizeof(cplx<R>);
  // the FP64 block of 256 sites takes 48 KB, which with the static reduction scratch
  // is above the default limit (set on the current device, every such launch)
  if (smem > 40 * 1024)
    WCMG_CUDA(cudaFuncSetAttribute(k_sap_fine<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sap_fine<R><<<dim3(nblocks, nrhs), nt, smem, st>>>(x, b, Dx, gauge, clov, g.V, bi, blocks, steps);
  WCMG_LAUNCH_CHECK();
}

// ---- C(x)^-1 (even-odd preconditioned SAP block solves) ----
// Per site and chirality half the 6x6 Hermitian block of C is inverted in FP64 by
// Gauss-Jordan elimination with partial pivoting; the inverse is Hermitian and is
// packed like C (three pairs of real diagonal entries, then the 15 entries above the
// diagonal).  err receives 1 when a pivot vanishes (a singular site block).
__global__ void k_clover_invert(double2* __restrict__ inv, const double2* __restrict__ clov, int V,
                                int* __restrict__ err) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= 2LL * V) return;
  const int h = (int)(t / V), s = (int)(t - (long long)h * V);
  double2 a[6][12];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 12; ++j) a[i][j] = make_double2(j == i + 6 ? 1.0 : 0.0, 0.0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double2 d = clov[(long long)(18 * h + k) * V + s];
    a[2 * k][2 * k] = make_double2(d.x, 0.0);
    a[2 * k + 1][2 * k + 1] = make_double2(d.y, 0.0);
  }
  int o = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) {
      const double2 c = clov[(long long)(18 * h + o++) * V + s];
      a[i][j] = c;
      a[j][i] = make_double2(c.x, -c.y);
    }
  for (int col = 0; col < 6; ++col) {
    int p = col;
    double best = a[col][col].x * a[col][col].x + a[col][col].y * a[col][col].y;
    for (int r = col + 1; r < 6; ++r) {
      const double m = a[r][col].x * a[r][col].x + a[r][col].y * a[r][col].y;
      if (m > best) { best = m; p = r; }
    }
    if (!(best > 0.0)) {
      *err = 1;
      return;
    }
    if (p != col)
      for (int j = 0; j < 12; ++j) {
        const double2 tmp = a[p][j];
        a[p][j] = a[col][j];
        a[col][j] = tmp;
      }
    const double2 pv = a[col][col];
    const double2 ip = make_double2(pv.x / best, -pv.y / best);  // 1 / pv
    for (int j = 0; j < 12; ++j) {
      const double2 v = a[col][j];
      a[col][j] = make_double2(v.x * ip.x - v.y * ip.y, v.x * ip.y + v.y * ip.x);
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const double2 f = a[r][col];
      for (int j = 0; j < 12; ++j) {
        const double2 v = a[col][j];
        a[r][j].x -= f.x * v.x - f.y * v.y;
        a[r][j].y -= f.x * v.y + f.y * v.x;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
    inv[(long long)(18 * h + k) * V + s] = make_double2(a[2 * k][6 + 2 * k].x, a[2 * k + 1][6 + 2 * k + 1].x);
  o = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j) inv[(long long)(18 * h + o++) * V + s] = a[i][6 + j];
}

void launch_clover_invert(double2* inv, const double2* clov, int V, int* err, cudaStream_t st) {
  k_clover_invert<<<nblk(2LL * V, 64), 64, 0, st>>>(inv, clov, V, err);
  WCMG_LAUNCH_CHECK();
}

// ---- even-odd preconditioned SAP colour pass on the fine level ----
// As k_sap_fine, but each block solve D_B e = r runs on the block's Schur complement on
// its odd sites (sites even or odd by the parity of x + y + z + t; interior hops join
// opposite parities): with H the interior hops,
//   r^_o = r_o - H_oe C_ee^-1 r_e;  e_o = MR_k(S; r^_o), S = C_oo - H_oe C_ee^-1 H_eo,
//   one step length per block;  e_e = C_ee^-1 (r_e - H_eo e_o).
// The hop kernels accumulate sum_hops without the factor -1/2 of D, so H f = -acc/2.
// Threads 0 .. bvol/2-1 take the even site of each x-pair of the block (local sites
// 2q, 2q+1; b0 is even), the others the odd site, so a warp holds one parity when
// bvol/2 is a multiple of 32.  One shared array holds the odd-site vector and the
// even-site intermediate at once (each phase reads one parity and writes the other).
// opar[B]: parity of block B's first site.
template <typename R>
__global__ void __launch_bounds__(SAP_FINE_T, sizeof(R) == 4 ? 2 : 1)
    k_sap_fine_eo(cplx<R>* __restrict__ x, const cplx<R>* __restrict__ b, const cplx<R>* __restrict__ Dx,
                  const cplx<R>* __restrict__ U, const cplx<R>* __restrict__ clov,
                  const cplx<R>* __restrict__ cinv, int V, BlockInfo bi, const int* __restrict__ blocks,
                  const unsigned char* __restrict__ opar, int steps) {
  using T = cplx<R>;
  extern __shared__ __align__(16) unsigned char sap_smem[];
  T* rs = reinterpret_cast<T*>(sap_smem);
  const int NT = blockDim.x;
  const int half = bi.bvol / 2;
  const int B = blocks[blockIdx.x];
  const bool valid = (int)threadIdx.x < bi.bvol;
  const bool even = (int)threadIdx.x < half;
  const int q = valid ? (even ? threadIdx.x : threadIdx.x - half) : 0;
  int l[4], st[4];
  st[0] = 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) st[k + 1] = st[k] * bi.b[k];
  int j;
  {
    // parity of the pair's first site 2q decides which of 2q, 2q+1 is even
    int loc = 2 * q, par = opar[B];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      par += loc % bi.b[k];
      loc /= bi.b[k];
    }
    j = 2 * q + (((par & 1) == 0) == even ? 0 : 1);
    loc = j;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      l[k] = loc % bi.b[k];
      loc /= bi.b[k];
    }
  }
  const int s = B * bi.bvol + j;
  const long long off = (long long)blockIdx.y * 12 * V;
  // sum of the interior hops at this thread's site from the vector in rs
  auto hops = [&](T (&acc)[1][12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[0][c] = czero<R>();
#define WCMG_SAP_HOP(MU)                                                                  \
  if (l[MU] < bi.b[MU] - 1) hop_at<R, MU, true, 1>(acc, rs, 0, NT, j + st[MU], U, V, s); \
  if (l[MU] > 0) hop_at<R, MU, false, 1>(acc, rs, 0, NT, j - st[MU], U, V, s - st[MU]);
    WCMG_SAP_HOP(0)
    WCMG_SAP_HOP(1)
    WCMG_SAP_HOP(2)
    WCMG_SAP_HOP(3)
#undef WCMG_SAP_HOP
  };
  // out = M in for the site's clover (or inverse clover) M
  auto site_mul = [&](T (&out)[1][12], const T (&in)[12], const cplx<R>* __restrict__ M) {
#pragma unroll
    for (int c = 0; c < 12; ++c) out[0][c] = czero<R>();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      T p[1][6];
#pragma unroll
      for (int i = 0; i < 6; ++i) p[0][i] = in[6 * h + i];
      clover_half<R, 1>(out, M, p, h, V, s);
    }
  };
  T v[12], e[12], acc[1][12];
  // r on this site; even threads keep r_e, odd threads turn it into r^_o below
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    T r = czero<R>();
    if (valid) {
      const long long o = off + (long long)c * V + s;
      r = Dx ? b[o] - Dx[o] : b[o];
    }
    v[c] = r;
    e[c] = czero<R>();
  }
  if (valid && even) {
    site_mul(acc, v, cinv);  // t = C_ee^-1 r_e
#pragma unroll
    for (int c = 0; c < 12; ++c) rs[c * NT + j] = acc[0][c];
  }
  __syncthreads();
  if (valid && !even) {
    hops(acc);  // r^_o = r_o - H t = r_o + acc / 2
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      v[c] = v[c] + R(0.5) * acc[0][c];
      rs[c * NT + j] = v[c];
    }
  }
  __syncthreads();
  __shared__ double scratch[(SAP_FINE_T / 32) * 3], red[3];
  for (int k = 0; k < steps; ++k) {
    if (valid && even) {
      // w' = C_ee^-1 (acc / 2) = -C_ee^-1 H_eo v
      hops(acc);
      T u[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) u[c] = R(0.5) * acc[0][c];
      T w[1][12];
      site_mul(w, u, cinv);
#pragma unroll
      for (int c = 0; c < 12; ++c) rs[c * NT + j] = w[0][c];
    }
    __syncthreads();
    R v3[3] = {R(0), R(0), R(0)};
    if (valid && !even) {
      // p = S v = C v - H w = C v - acc / 2 with acc the hops of w' = -w
      hops(acc);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        T p[1][6];
#pragma unroll
        for (int i = 0; i < 6; ++i) p[0][i] = v[6 * h + i];
        clover_half<R, 1>(acc, clov, p, h, V, s);
      }
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        const T o = acc[0][c];
        v3[0] += o.x * v[c].x + o.y * v[c].y;
        v3[1] += o.x * v[c].y - o.y * v[c].x;
        v3[2] += o.x * o.x + o.y * o.y;
      }
    }
    block_sum_mixed<R, 3>(v3, scratch, red);
    const double pp = red[2];
    const T a = pp != 0.0 ? cmk((R)(red[0] / pp), (R)(red[1] / pp)) : czero<R>();
    if (valid && !even) {
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        cmac(e[c], a, v[c]);
        v[c] = v[c] - cmul(a, acc[0][c]);
        rs[c * NT + j] = v[c];
      }
    }
    __syncthreads();
  }
  if (valid && !even) {
#pragma unroll
    for (int c = 0; c < 12; ++c) rs[c * NT + j] = e[c];
  }
  __syncthreads();
  if (valid && even) {
    // e_e = C_ee^-1 (r_e - H e_o) = C_ee^-1 (r_e + acc / 2)
    hops(acc);
    T u[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) u[c] = v[c] + R(0.5) * acc[0][c];
    T w[1][12];
    site_mul(w, u, cinv);
#pragma unroll
    for (int c = 0; c < 12; ++c) e[c] = w[0][c];
  }
  if (valid) {
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const long long o = off + (long long)c * V + s;
      x[o] = x[o] + e[c];
    }
  }
}

template <typename R>
void launch_sap_fine_eo(cplx<R>* x, const cplx<R>* b, const cplx<R>* Dx, const cplx<R>* gauge, const cplx<R>* clov,
                        const cplx<R>* cinv, const LevelGeom& g, const int* blocks, const unsigned char* opar,
                        int nblocks, int steps, int nrhs, cudaStream_t st) {
  const int nt = sap_fine_threads(g.bvol);
  if (!nt || (g.b[0] & 1)) throw Error(-1, "even-odd SAP pass needs aggregates of <= 256 sites, even in x");
  if (nblocks <= 0) return;
  BlockInfo bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const size_t smem = (size_t)12 * nt * sizeof(cplx<R>);
  if (smem > 40 * 1024)
    WCMG_CUDA(cudaFuncSetAttribute(k_sap_fine_eo<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_sap_fine_eo<R><<<dim3(nblocks, nrhs), nt, smem, st>>>(x, b, Dx, gauge, clov, cinv, g.V, bi, blocks, opar, steps);
  WCMG_LAUNCH_CHECK();
}

// ---- chirality pairs for CoarsenOperator (K5) ----
// For each near-null vector v_i the Galerkin construction needs the masked stencil
// applied to both chirality projections: out[i] = D_mode(Pi_+ v_i),
// out[nv + i] = D_mode(Pi_- v_i).  Pi_+ v keeps spin 0, 1 and Pi_- v spin 2, 3
// (chiral basis), so one load of v's neighbour spinor serves both: the projected
// half spinor of Pi_+ v is its upper half, that of Pi_- v is -/+ B of its lower
// half.  The clover term is chirality-diagonal: C Pi_+ v = C_upper acting on the
// upper half only.
template <typename R, int MU, bool FWD>
__device__ __forceinline__ void hop_chiral(cplx<R> (&ap)[12], cplx<R> (&am)[12], const cplx<R>* __restrict__ in,
                                           const cplx<R>* __restrict__ U, int V, int s, int y) {
  using T = cplx<R>;
  const int ls = FWD ? s : y;
  T u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = U[((long long)MU * 9 + k) * V + ls];
  T hp[2][3], pl[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      hp[sp][c] = in[(long long)(3 * sp + c) * V + y];
      pl[sp][c] = in[(long long)(6 + 3 * sp + c) * V + y];
    }
  T hm[2][3];
  applyB<MU>(hm, pl);
  if (FWD) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int c = 0; c < 3; ++c) hm[sp][c] = -hm[sp][c];
  }
  T wp[2][3], wm[2][3];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T tp = czero<R>(), tm = czero<R>();
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (FWD) {
          cmac(tp, u[3 * a + b], hp[sp][b]);
          cmac(tm, u[3 * a + b], hm[sp][b]);
        } else {
          cjmac(tp, u[3 * b + a], hp[sp][b]);
          cjmac(tm, u[3 * b + a], hm[sp][b]);
        }
      }
      wp[sp][a] = tp;
      wm[sp][a] = tm;
    }
  T Bp[2][3], Bm[2][3];
  applyBdag<MU>(Bp, wp);
  applyBdag<MU>(Bm, wm);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ap[3 * sp + c] += wp[sp][c];
      am[3 * sp + c] += wm[sp][c];
      if (FWD) {
        ap[6 + 3 * sp + c] -= Bp[sp][c];
        am[6 + 3 * sp + c] -= Bm[sp][c];
      } else {
        ap[6 + 3 * sp + c] += Bp[sp][c];
        am[6 + 3 * sp + c] += Bm[sp][c];
      }
    }
}

template <typename R, int MODE>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1)
    k_dslash_chiral(cplx<R>* __restrict__ out, const cplx<R>* __restrict__ in, const cplx<R>* __restrict__ U,
                    const cplx<R>* __restrict__ clov, const int* __restrict__ nbr, int V, BlockInfo bi, int hopdir,
                    int nv) {
  using T = cplx<R>;
  const int i = blockIdx.x % nv;  // vector fastest: the CTAs running together share links and clover
  const int t = (blockIdx.x / nv) * blockDim.x + threadIdx.x;
  int s = t;
  if (MODE == ST_FACE_HOP) {
    // one thread per site of the hopdir face of every aggregate: face site f of block
    // t / nface has l[mu] fixed and the other local coordinates from f (x fastest)
    const int mu = hopdir >> 1, nface = bi.bvol / bi.b[mu];
    if (t >= V / bi.b[mu]) return;
    int f = t % nface, loc = 0, stride = 1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int lk;
      if (k == mu) {
        lk = (hopdir & 1) ? 0 : bi.b[mu] - 1;
      } else {
        lk = f % bi.b[k];
        f /= bi.b[k];
      }
      loc += lk * stride;
      stride *= bi.b[k];
    }
    s = (t / nface) * bi.bvol + loc;
  } else if (s >= V) {
    return;
  }
  const long long rstride = 12LL * V;
  const cplx<R>* vi = in + (long long)i * rstride;
  T ap[12], am[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) ap[c] = am[c] = czero<R>();
  auto use = [&](int d) -> bool {
    if (MODE == ST_BLOCK_INTERIOR) return !on_face(bi, s, d);
    return d == hopdir && on_face(bi, s, d);
  };
#define WCMG_HOPC(MU)                                                                       \
  if (use(2 * MU)) hop_chiral<R, MU, true>(ap, am, vi, U, V, s, nbr[(2 * MU) * V + s]);      \
  if (use(2 * MU + 1)) hop_chiral<R, MU, false>(ap, am, vi, U, V, s, nbr[(2 * MU + 1) * V + s]);
  WCMG_HOPC(0)
  WCMG_HOPC(1)
  WCMG_HOPC(2)
  WCMG_HOPC(3)
#undef WCMG_HOPC
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    ap[c] = R(-0.5) * ap[c];
    am[c] = R(-0.5) * am[c];
  }
  if (MODE != ST_FACE_HOP) {
    // C Pi_+ v: upper 6x6 block on the upper half; C Pi_- v: lower block on the lower half
    T p[1][6];
    T accp[1][12], accm[1][12];
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      accp[0][c] = R(-2.0) * ap[c];  // clover_half computes C p - acc / 2 on its half
      accm[0][c] = R(-2.0) * am[c];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) p[0][k] = vi[(long long)k * V + s];
    clover_half<R, 1>(accp, clov, p, 0, V, s);
#pragma unroll
    for (int k = 0; k < 6; ++k) p[0][k] = vi[(long long)(6 + k) * V + s];
    clover_half<R, 1>(accm, clov, p, 1, V, s);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ap[k] = accp[0][k];
      am[6 + k] = accm[0][6 + k];
    }
  }
  T* op = out + (long long)i * rstride;
  T* om = out + (long long)(nv + i) * rstride;
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    op[(long long)c * V + s] = ap[c];
    om[(long long)c * V + s] = am[c];
  }
}

template <typename R>
void launch_dslash_chiral(cplx<R>* out, const cplx<R>* vecs, const cplx<R>* gauge, const cplx<R>* clov,
                          const LevelGeom& g, int nv, int mode, int hopdir, cudaStream_t st) {
  BlockInfo bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  if (mode == ST_BLOCK_INTERIOR) {
    const dim3 grid((unsigned)(nblk(g.V, 128) * (long long)nv));
    k_dslash_chiral<R, ST_BLOCK_INTERIOR><<<grid, 128, 0, st>>>(out, vecs, gauge, clov, g.nbr, g.V, bi, hopdir, nv);
  } else if (mode == ST_FACE_HOP) {
    if (hopdir < 0 || hopdir > 7) throw Error(-1, "chirality-pair stencil: face direction out of range");
    const dim3 grid((unsigned)(nblk(g.V / g.b[hopdir >> 1], 128) * (long long)nv));
    k_dslash_chiral<R, ST_FACE_HOP><<<grid, 128, 0, st>>>(out, vecs, gauge, clov, g.nbr, g.V, bi, hopdir, nv);
  }
  else
    throw Error(-1, "chirality-pair stencil: block-interior or face mode only");
  WCMG_LAUNCH_CHECK();
}

// pr[r] = sum_b pr_part[r][b], pp[r] = sum_b pp_part[r][b] (fixed tree)
__global__ void __launch_bounds__(256) k_mr_final(double2* __restrict__ pr, double* __restrict__ pp,
                                                  const double2* __restrict__ pr_part,
                                                  const double* __restrict__ pp_part, int nsb) {
  __shared__ double scratch[(256 / 32) * 3];
  __shared__ double red[3];
  const int r = blockIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nsb; b += 256) {
    const double2 a = pr_part[(long long)r * nsb + b];
    v[0] += a.x;
    v[1] += a.y;
    v[2] += pp_part[(long long)r * nsb + b];
  }
  block_sum_regs<double, 3>(v, 3, scratch, red);
  if (threadIdx.x == 0) {
    pr[r] = make_double2(red[0], red[1]);
    pp[r] = red[2];
  }
}

int dslash_partials(int V) { return (int)nblk(V, 128); }

template <typename R>
void launch_dslash_mr(cplx<R>* out, const cplx<R>* in, const cplx<R>* gauge, const cplx<R>* clov, const LevelGeom& g,
                      int nrhs, double2* pr, double* pp, double2* pr_part, double* pp_part, cudaStream_t st) {
  BlockInfo bi;
  for (int k = 0; k < 4; ++k) bi.b[k] = g.b[k];
  bi.bvol = g.bvol;
  const int nsb = dslash_partials(g.V);
  const int nr = dslash_nr<R>(nrhs);
  const unsigned grid = (unsigned)((long long)nsb * ((nrhs + nr - 1) / nr));
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    if (nr == 2) {
      k_dslash<R, ST_FULL, true, 2><<<grid, 128, 0, st>>>(out, in, gauge, clov, g.nbr, g.V, bi, 0, nrhs, pr_part,
                                                           pp_part, nullptr, 0);
      done = true;
    }
  }
  if (!done)
    k_dslash<R, ST_FULL, true, 1><<<grid, 128, 0, st>>>(out, in, gauge, clov, g.nbr, g.V, bi, 0, nrhs, pr_part,
                                                         pp_part, nullptr, 0);
  WCMG_LAUNCH_CHECK();
  k_mr_final<<<nrhs, 256, 0, st>>>(pr, pp, pr_part, pp_part, nsb);
  WCMG_LAUNCH_CHECK();
}

#define WCMG_INST(R)                                                                                          \
  template void launch_pack_fine<R>(cplx<R>*, const double2*, const int*, int, int, cudaStream_t);            \
  template void launch_unpack_fine<R>(double2*, const cplx<R>*, const int*, int, int, cudaStream_t);          \
  template void launch_pack_gauge<R>(cplx<R>*, const double2*, const int*, int, cudaStream_t);                \
  template void launch_dslash<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*, const LevelGeom&, \
                                 int, int, int, cudaStream_t, const unsigned char*, int);                    \
  template void launch_sap_fine<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*,  \
                                   const LevelGeom&, const int*, int, int, int, cudaStream_t);                \
  template void launch_sap_fine_eo<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*,              \
                                      const cplx<R>*, const cplx<R>*, const LevelGeom&, const int*,           \
                                      const unsigned char*, int, int, int, cudaStream_t);                     \
  template void launch_dslash_mr<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*, const LevelGeom&, \
                                    int, double2*, double*, double2*, double*, cudaStream_t);                  \
  template void launch_dslash_chiral<R>(cplx<R>*, const cplx<R>*, const cplx<R>*, const cplx<R>*,              \
                                        const LevelGeom&, int, int, int, cudaStream_t);
WCMG_INST(double)
WCMG_INST(float)
#undef WCMG_INST

}  // namespace wcmg
