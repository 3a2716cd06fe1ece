// Gauge-equivariant parallel-transport convolution (PTC) network kernels: the
// learned coarse correction.  The paper has no learned component; the network
// maps a fine residual to an approximation of the multigrid coarse-grid
// correction P D_c^-1 P^dag r built from the operators of Sec. 2.1.
//
//   layer:  out_i(x) = sum_j sum_h W_{ijh} (T_h in_j)(x)
//   hops:   h = 0 identity, 1 + 2 mu: (T f)(x) = U_mu(x) f(x + mu),
//           2 + 2 mu: (T f)(x) = U_mu(x - mu)^dag f(x - mu);  T_{+-mu}^dag = T_{-+mu}
//   W_{ijh} complex 4x4 spin matrices (spin index), T_h acts on colour.
// Fields use the fine layout [12][V] (component 3 * spin + colour), FP32.
// Every kernel recomputes the transports on the fly (one SU(3) matvec per spin
// and hop) instead of storing nin x 9 transported fields.
#include "kernels.h"

namespace wcmg {

constexpr int PTC_NHOP = 9;

// t = (T_h f)(x), 12 complex, FP32
__device__ __forceinline__ void ptc_transport(float2 (&t)[12], const float2* __restrict__ f,
                                              const float2* __restrict__ U, const int* __restrict__ nbr, int V, int x,
                                              int h) {
  if (h == 0) {
#pragma unroll
    for (int c = 0; c < 12; ++c) t[c] = f[(long long)c * V + x];
    return;
  }
  const int mu = (h - 1) >> 1, back = (h - 1) & 1;
  const int y = nbr[(2 * mu + back) * V + x];
  const int ls = back ? y : x;
  float2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = U[((long long)mu * 9 + k) * V + ls];
  float2 g[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) g[c] = f[(long long)c * V + y];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (!back) cmac(acc, u[3 * a + b], g[3 * s + b]);
        else cjmac(acc, u[3 * b + a], g[3 * s + b]);
      }
      t[3 * s + a] = acc;
    }
}

// opposite hop: T_h^dag = T_{opp(h)}
__device__ __forceinline__ int ptc_opp(int h) { return h == 0 ? 0 : (((h - 1) & 1) ? h - 1 : h + 1); }

// Forward layer.  Thread per (site, output channel i, rhs); W in shared memory.
// Each thread computes OG output fields at its site: the parallel transport of an
// input field along a hop is formed once and applied to the OG spin weights (every
// output still sums its terms in the same order).
template <int OG>
__global__ void __launch_bounds__(128) k_ptc_forward(float2* __restrict__ out, const float2* __restrict__ in,
                                                     const float2* __restrict__ W, const float2* __restrict__ U,
                                                     const int* __restrict__ nbr, int V, int nin, int nout, int nrhs) {
  extern __shared__ float2 Ws[];
  const int nw = nout * nin * PTC_NHOP * 16;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) Ws[k] = W[k];
  __syncthreads();
  const int ngrp = (nout + OG - 1) / OG;
  const int io0 = (blockIdx.y % ngrp) * OG, r = blockIdx.y / ngrp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V || r >= nrhs) return;
  const long long fs = 12LL * V;
  float2 acc[OG][12];
#pragma unroll
  for (int g = 0; g < OG; ++g)
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[g][c] = make_float2(0.f, 0.f);
  for (int j = 0; j < nin; ++j) {
    const float2* f = in + ((long long)r * nin + j) * fs;
    for (int h = 0; h < PTC_NHOP; ++h) {
      float2 t[12];
      ptc_transport(t, f, U, nbr, V, x, h);
#pragma unroll
      for (int g = 0; g < OG; ++g) {
        if (io0 + g >= nout) break;
        const float2* w = Ws + (((io0 + g) * nin + j) * PTC_NHOP + h) * 16;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const float2 wab = w[4 * a + b];
#pragma unroll
            for (int c = 0; c < 3; ++c) cmac(acc[g][3 * a + c], wab, t[3 * b + c]);
          }
      }
    }
  }
#pragma unroll
  for (int g = 0; g < OG; ++g) {
    if (io0 + g >= nout) break;
    float2* o = out + ((long long)r * nout + io0 + g) * fs;
#pragma unroll
    for (int c = 0; c < 12; ++c) o[(long long)c * V + x] = acc[g][c];
  }
}

// Backward with respect to the layer input:
//   gin_j(x) = sum_h T_h^dag ( sum_i W_{ijh}^dag g_i )(x),
// with T_h^dag = T_{opp(h)}: the spin-mixed gradient is formed at the neighbour
// site the adjoint hop reads from, then transported.
__global__ void __launch_bounds__(128) k_ptc_backward_data(float2* __restrict__ gin, const float2* __restrict__ gout,
                                                           const float2* __restrict__ W,
                                                           const float2* __restrict__ U,
                                                           const int* __restrict__ nbr, int V, int nin, int nout,
                                                           int nrhs) {
  extern __shared__ float2 Ws[];
  const int nw = nout * nin * PTC_NHOP * 16;
  for (int k = threadIdx.x; k < nw; k += blockDim.x) Ws[k] = W[k];
  __syncthreads();
  const int j = blockIdx.y % nin, r = blockIdx.y / nin;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V || r >= nrhs) return;
  const long long fs = 12LL * V;
  float2 acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = make_float2(0.f, 0.f);
  for (int h = 0; h < PTC_NHOP; ++h) {
    const int ho = ptc_opp(h);
    // site y the adjoint hop reads from and the link it applies
    int y = x;
    int mu = 0, back = 0;
    if (ho != 0) {
      mu = (ho - 1) >> 1;
      back = (ho - 1) & 1;
      y = nbr[(2 * mu + back) * V + x];
    }
    float2 s[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) s[c] = make_float2(0.f, 0.f);
    for (int i = 0; i < nout; ++i) {
      const float2* g = gout + ((long long)r * nout + i) * fs;
      float2 gy[12];
#pragma unroll
      for (int c = 0; c < 12; ++c) gy[c] = g[(long long)c * V + y];
      const float2* w = Ws + ((i * nin + j) * PTC_NHOP + h) * 16;
      // s[b][c] += sum_a conj(W[a][b]) g[a][c]
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float2 wab = w[4 * a + b];
#pragma unroll
          for (int c = 0; c < 3; ++c) cjmac(s[3 * b + c], wab, gy[3 * a + c]);
        }
    }
    if (ho == 0) {
#pragma unroll
      for (int c = 0; c < 12; ++c) acc[c] += s[c];
    } else {
      const int ls = back ? y : x;
      float2 u[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) u[k] = U[((long long)mu * 9 + k) * V + ls];
#pragma unroll
      for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            if (!back) cmac(acc[3 * sp + a], u[3 * a + b], s[3 * sp + b]);
            else cjmac(acc[3 * sp + a], u[3 * b + a], s[3 * sp + b]);
          }
    }
  }
  float2* o = gin + ((long long)r * nin + j) * fs;
#pragma unroll
  for (int c = 0; c < 12; ++c) o[(long long)c * V + x] = acc[c];
}

// Weight gradient, first stage: per warp (32 sites of one rhs) and per
// (i, j, h), the 16 entries sum_{x,c} g_i[a][c](x) conj((T_h in_j)[b][c](x)),
// reduced by warp shuffles; partial[(warp_global)][(i j h a b)].
__global__ void __launch_bounds__(128) k_ptc_wgrad_partial(float2* __restrict__ partial,
                                                           const float2* __restrict__ gout,
                                                           const float2* __restrict__ in,
                                                           const float2* __restrict__ U,
                                                           const int* __restrict__ nbr, int V, int nin, int nout,
                                                           int nrhs) {
  const int lane = threadIdx.x & 31;
  const int wpr = (V + 31) / 32;  // warps per rhs
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (wg >= (long long)wpr * nrhs) return;
  const int r = (int)(wg / wpr), x = (int)(wg % wpr) * 32 + lane;
  const bool valid = x < V;
  const int xs = valid ? x : 0;
  const long long fs = 12LL * V;
  const int nent = nout * nin * PTC_NHOP * 16;
  float2* part = partial + wg * nent;
  for (int j = 0; j < nin; ++j) {
    const float2* f = in + ((long long)r * nin + j) * fs;
    for (int h = 0; h < PTC_NHOP; ++h) {
      float2 t[12];
      ptc_transport(t, f, U, nbr, V, xs, h);
      if (!valid) {
#pragma unroll
        for (int c = 0; c < 12; ++c) t[c] = make_float2(0.f, 0.f);
      }
      for (int i = 0; i < nout; ++i) {
        const float2* g = gout + ((long long)r * nout + i) * fs;
        float2 gx[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) gx[c] = valid ? g[(long long)c * V + xs] : make_float2(0.f, 0.f);
        float2 vals[16];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) cjmac(v, t[3 * b + c], gx[3 * a + c]);  // g conj(t)
            vals[4 * a + b] = v;
          }
#pragma unroll
        for (int k = 0; k < 16; ++k) vals[k] = warp_sum(vals[k]);
        if (lane < 16) {
          float2 v = vals[0];
#pragma unroll
          for (int k = 1; k < 16; ++k)
            if (lane == k) v = vals[k];
          part[((i * nin + j) * PTC_NHOP + h) * 16 + lane] = v;
        }
      }
    }
  }
}

// second stage: gW[e] = sum_w partial[w][e] (fixed order)
__global__ void k_ptc_wgrad_final(float2* __restrict__ gW, const float2* __restrict__ partial, long long nwarps,
                                  int nent) {
  __shared__ double2 scratch[8];
  __shared__ double2 red[1];
  const int e = blockIdx.x;
  double2 acc = make_double2(0, 0);
  for (long long w = threadIdx.x; w < nwarps; w += blockDim.x) {
    const float2 v = partial[w * nent + e];
    acc.x += v.x;
    acc.y += v.y;
  }
  block_sum_many<double2>(&acc, 1, scratch, red);
  if (threadIdx.x == 0) gW[e] = make_float2((float)red[0].x, (float)red[0].y);
}

// Adam on the real and imaginary parts (real gradient = 2 x Wirtinger gradient).
__global__ void k_ptc_adam(float2* __restrict__ w, const float2* __restrict__ g, float2* __restrict__ m,
                           float2* __restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1,
                           float bc2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float2 gr = make_float2(2.f * g[k].x, 2.f * g[k].y);
  float2 mk = m[k], vk = v[k];
  mk.x = b1 * mk.x + (1.f - b1) * gr.x;
  mk.y = b1 * mk.y + (1.f - b1) * gr.y;
  vk.x = b2 * vk.x + (1.f - b2) * gr.x * gr.x;
  vk.y = b2 * vk.y + (1.f - b2) * gr.y * gr.y;
  m[k] = mk;
  v[k] = vk;
  float2 wk = w[k];
  wk.x -= lr * (mk.x / bc1) / (sqrtf(vk.x / bc2) + eps);
  wk.y -= lr * (mk.y / bc1) / (sqrtf(vk.y / bc2) + eps);
  w[k] = wk;
}

// Counter-based Gaussian field (SplitMix64 finaliser on seed * phi + stream * c +
// index, uniform from the top 53 bits, Box-Muller), the same generator as the
// host-side input module, drawn on the device for training residuals.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long stream, unsigned long long i) {
  const unsigned long long c = seed * 0x9E3779B97F4A7C15ULL + stream * 0xD1B54A32D192ED03ULL + i;
  return (double)(splitmix64(c) >> 11) * (1.0 / 9007199254740992.0);
}
__global__ void k_gaussian_field(float2* __restrict__ out, long long n, unsigned long long seed,
                                 unsigned long long stream) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double u1 = u01(seed, stream, 2 * i), u2 = u01(seed, stream, 2 * i + 1);
  const double rad = sqrt(-2.0 * log1p(-u1));
  double sv, cv;
  sincospi(2.0 * u2, &sv, &cv);
  out[i] = make_float2((float)(rad * cv), (float)(rad * sv));
}

// ---------------- launchers ----------------
void launch_ptc_forward(float2* out, const float2* in, const float2* W, const float2* U, const int* nbr, int V,
                        int nin, int nout, int nrhs, cudaStream_t st) {
  const size_t smem = (size_t)nout * nin * PTC_NHOP * 16 * sizeof(float2);
  if (nout >= 4)
    k_ptc_forward<4><<<dim3(nblk(V, 128), ((nout + 3) / 4) * nrhs), 128, smem, st>>>(out, in, W, U, nbr, V, nin,
                                                                                     nout, nrhs);
  else
    k_ptc_forward<1><<<dim3(nblk(V, 128), nout * nrhs), 128, smem, st>>>(out, in, W, U, nbr, V, nin, nout, nrhs);
  WCMG_LAUNCH_CHECK();
}
void launch_ptc_backward_data(float2* gin, const float2* gout, const float2* W, const float2* U, const int* nbr, int V,
                              int nin, int nout, int nrhs, cudaStream_t st) {
  const size_t smem = (size_t)nout * nin * PTC_NHOP * 16 * sizeof(float2);
  k_ptc_backward_data<<<dim3(nblk(V, 128), nin * nrhs), 128, smem, st>>>(gin, gout, W, U, nbr, V, nin, nout, nrhs);
  WCMG_LAUNCH_CHECK();
}
long long ptc_wgrad_partial_size(int V, int nin, int nout, int nrhs) {
  return (long long)((V + 31) / 32) * nrhs * nout * nin * PTC_NHOP * 16;
}
void launch_ptc_wgrad(float2* gW, float2* partial, const float2* gout, const float2* in, const float2* U,
                      const int* nbr, int V, int nin, int nout, int nrhs, cudaStream_t st) {
  const long long nwarps = (long long)((V + 31) / 32) * nrhs;
  k_ptc_wgrad_partial<<<(unsigned)((nwarps + 3) / 4), 128, 0, st>>>(partial, gout, in, U, nbr, V, nin, nout, nrhs);
  WCMG_LAUNCH_CHECK();
  const int nent = nout * nin * PTC_NHOP * 16;
  k_ptc_wgrad_final<<<nent, 256, 0, st>>>(gW, partial, nwarps, nent);
  WCMG_LAUNCH_CHECK();
}
void launch_ptc_adam(float2* w, const float2* g, float2* m, float2* v, int n, float lr, int t, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  k_ptc_adam<<<nblk(n, 256), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, 1e-8f, 1.f - powf(b1, (float)t),
                                           1.f - powf(b2, (float)t));
  WCMG_LAUNCH_CHECK();
}
void launch_gaussian_field(float2* out, long long n, unsigned long long seed, unsigned long long stream,
                           cudaStream_t st) {
  k_gaussian_field<<<nblk(n, 256), 256, 0, st>>>(out, n, seed, stream);
  WCMG_LAUNCH_CHECK();
}

}  // namespace wcmg
