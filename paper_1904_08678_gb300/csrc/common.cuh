// Shared device helpers of the wcmg kernels: complex arithmetic on double2 /
// float2, link storage conversions, warp/block reductions, error plumbing.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <stdexcept>
#include <string>

namespace wcmg {

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename R> using cplx = typename cplx_of<R>::type;

__host__ __device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
template <typename R> __host__ __device__ __forceinline__ cplx<R> czero() { return cmk(R(0), R(0)); }

#define WCMG_CPLX_OPS(T, R)                                                                         \
  __host__ __device__ __forceinline__ T operator+(T a, T b) { return cmk(a.x + b.x, a.y + b.y); }   \
  __host__ __device__ __forceinline__ T operator-(T a, T b) { return cmk(a.x - b.x, a.y - b.y); }   \
  __host__ __device__ __forceinline__ T operator-(T a) { return cmk(-a.x, -a.y); }                  \
  __host__ __device__ __forceinline__ T operator*(R s, T a) { return cmk(s * a.x, s * a.y); }       \
  __host__ __device__ __forceinline__ T& operator+=(T& a, T b) { a.x += b.x; a.y += b.y; return a; } \
  __host__ __device__ __forceinline__ T& operator-=(T& a, T b) { a.x -= b.x; a.y -= b.y; return a; } \
  /* a * b */                                                                                       \
  __host__ __device__ __forceinline__ T cmul(T a, T b) {                                            \
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                                       \
  }                                                                                                 \
  /* conj(a) * b */                                                                                 \
  __host__ __device__ __forceinline__ T cjmul(T a, T b) {                                           \
    return cmk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);                                       \
  }                                                                                                 \
  /* acc += a * b */                                                                                \
  __host__ __device__ __forceinline__ void cmac(T& acc, T a, T b) {                                 \
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);                                    \
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);                                     \
  }                                                                                                 \
  /* acc += conj(a) * b */                                                                          \
  __host__ __device__ __forceinline__ void cjmac(T& acc, T a, T b) {                                \
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);                                     \
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);                                    \
  }                                                                                                 \
  /* acc -= a * b  (four fused multiply-adds) */                                                    \
  __host__ __device__ __forceinline__ void cnmac(T& acc, T a, T b) {                                \
    acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);                                    \
    acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);                                   \
  }                                                                                                 \
  __host__ __device__ __forceinline__ T conjg(T a) { return cmk(a.x, -a.y); }                       \
  /* i * a, -i * a */                                                                               \
  __host__ __device__ __forceinline__ T mul_i(T a) { return cmk(-a.y, a.x); }                       \
  __host__ __device__ __forceinline__ T mul_mi(T a) { return cmk(a.y, -a.x); }                      \
  __host__ __device__ __forceinline__ R cnorm2(T a) { return a.x * a.x + a.y * a.y; }

WCMG_CPLX_OPS(double2, double)
WCMG_CPLX_OPS(float2, float)
#undef WCMG_CPLX_OPS

__host__ __device__ __forceinline__ double2 to_c64(double2 a) { return a; }
__host__ __device__ __forceinline__ double2 to_c64(float2 a) { return make_double2(a.x, a.y); }
template <typename R> __host__ __device__ __forceinline__ cplx<R> from_c64(double2 a);
template <> __host__ __device__ __forceinline__ double2 from_c64<double>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 from_c64<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// ---- coarse-link storage types: complex numbers stored as (re, im) pairs ----
struct bf16c { __nv_bfloat162 v; };
struct f16c { __half2 v; };

template <typename L, typename R> __device__ __forceinline__ cplx<R> link_load(const L& l);
template <> __device__ __forceinline__ double2 link_load<double2, double>(const double2& l) { return l; }
template <> __device__ __forceinline__ float2 link_load<float2, float>(const float2& l) { return l; }
template <> __device__ __forceinline__ float2 link_load<bf16c, float>(const bf16c& l) { return __bfloat1622float2(l.v); }
template <> __device__ __forceinline__ float2 link_load<f16c, float>(const f16c& l) { return __half22float2(l.v); }

template <typename L> __device__ __forceinline__ L link_store(double2 a);
template <> __device__ __forceinline__ double2 link_store<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 link_store<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <> __device__ __forceinline__ bf16c link_store<bf16c>(double2 a) {
  bf16c r; r.v = __floats2bfloat162_rn((float)a.x, (float)a.y); return r;
}
template <> __device__ __forceinline__ f16c link_store<f16c>(double2 a) {
  f16c r; r.v = __floats2half2_rn((float)a.x, (float)a.y); return r;
}

// ---- reductions (fixed order: deterministic for fixed launch shapes) ----
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }
__device__ __forceinline__ float2 warp_sum(float2 v) { return make_float2(warp_sum(v.x), warp_sum(v.y)); }

__device__ __forceinline__ double2 shfl_xor2(double2 v, int o) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 shfl_xor2(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Warp sums of 8 values at once by a transposing butterfly: at each of the first
// three exchange steps (lane distance 16, 8, 4) a lane keeps half of its values
// and adds its partner's copy of that half, so 8 values cost 7 + 2 additions per
// lane instead of 8 x 5.  On return v[0] of lane l holds the full warp sum of
// value 4 b4 + 2 b3 + b2 (b_i: bit i of l); lanes with (l & 3) == 0 hold distinct
// values.
template <typename T>
__device__ __forceinline__ void warp_sum8_transposed(T (&v)[8], int lane) {
  {
    const bool up = lane & 16;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T send = up ? v[j] : v[j + 4];
      const T keep = up ? v[j + 4] : v[j];
      v[j] = keep + shfl_xor2(send, 16);
    }
  }
  {
    const bool up = lane & 8;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const T send = up ? v[j] : v[j + 2];
      const T keep = up ? v[j + 2] : v[j];
      v[j] = keep + shfl_xor2(send, 8);
    }
  }
  {
    const bool up = lane & 4;
    const T send = up ? v[0] : v[1];
    const T keep = up ? v[1] : v[0];
    v[0] = keep + shfl_xor2(send, 4);
  }
  v[0] += shfl_xor2(v[0], 2);
  v[0] += shfl_xor2(v[0], 1);
}
// index of the value that lane l holds after warp_sum8_transposed
__device__ __forceinline__ int warp_sum8_index(int lane) {
  return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Block sums of N real values: warp sums in the working precision R (FP32 shuffles
// and adds are cheap; FP64 adds run at 1/64 of the FP32 rate on this part), then
// FP64 across the warps.  Result k in red[k]; scratch holds (blockDim/32) * N.
template <typename R, int N>
__device__ __forceinline__ void block_sum_mixed(const R (&vals)[N], double* scratch, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const R s = warp_sum(vals[k]);
    if (lane == 0) scratch[warp * N + k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double t = scratch[threadIdx.x];
    for (int w = 1; w < nw; ++w) t += scratch[w * N + threadIdx.x];
    red[threadIdx.x] = t;
  }
  __syncthreads();
}

// Sum `n` complex values held per thread across the whole block; result for value k
// is left in red[k] (shared, size >= n).  scratch must hold (blockDim/32) * n values.
template <typename T>
__device__ __forceinline__ void block_sum_many(T* vals, int n, T* scratch, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    T s = warp_sum(vals[k]);
    if (lane == 0) scratch[warp * n + k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T s = scratch[k];
    for (int w = 1; w < nw; ++w) s += scratch[w * n + k];
    red[k] = s;
  }
  __syncthreads();
}

// Register-resident variant: vals has a compile-time size N (fully unrolled, so
// the array stays in registers); the first n entries are summed into red[0..n).
// scratch must hold (blockDim/32) * N values.
template <typename T, int N>
__device__ __forceinline__ void block_sum_regs(const T (&vals)[N], int n, T* scratch, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k < n) {
      T s = warp_sum(vals[k]);
      if (lane == 0) scratch[warp * N + k] = s;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    T s = scratch[k];
    for (int w = 1; w < nw; ++w) s += scratch[w * N + k];
    red[k] = s;
  }
  __syncthreads();
}

// ---- TMA bulk copies and mbarriers (inline PTX, sm_90+ / sm_103a) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also announces `bytes` of transaction to complete the phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase: gives up after `limit` polls (returns false).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = (1LL << 26)) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// ---- tcgen05 (5th-generation tensor cores, TMEM accumulators) ----
// Shared-memory matrix descriptor for a no-swizzle K-major operand: core
// matrices of 8 rows x 16 bytes; lbo = byte distance of K-adjacent core
// matrices, sbo = byte distance of row-adjacent (8-row) core matrices.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 generation; base offset 0, no swizzle
  return d;
}
// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 32 lanes x 16 columns of FP32 from TMEM (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- host-side error plumbing ----
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define WCMG_CUDA(call)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      throw ::wcmg::Error(e_ == cudaErrorMemoryAllocation ? -7 : -2,                             \
                          std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

// Number of kernels this library has launched (host side, one process).
inline long long& launch_counter() {
  static long long n = 0;
  return n;
}
#define WCMG_LAUNCH_CHECK()          \
  do {                               \
    ++::wcmg::launch_counter();      \
    WCMG_CUDA(cudaGetLastError());   \
  } while (0)

inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace wcmg
