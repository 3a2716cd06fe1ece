// Allocation-free entry point: block orthonormalisation of fine-level
// near-null vectors without a context and without any device allocation.
//
// Some callers cannot allocate device memory: their device memory is owned by
// another allocator (for example a host framework's caching pool) and they must
// not call cudaMalloc / cudaFree, which synchronise the whole device and can
// fail at run time once the pool holds the memory.  This entry point takes the
// caller's input and output buffers and keeps its own working copy in a
// file-scope device array of fixed size.
#include <mutex>

#include "../../include/wcmg.h"
#include "kernels.h"

namespace wcmg {
namespace {

constexpr long long kMaxElems = WCMG_NOALLOC_MAX_ELEMS;

// Working copy of the vectors in the library's internal fine layout
// ([nvec][12][V], aggregate-major sites), followed by the rank-check word.
// Host code must not use this name as a device address: it is looked up once
// per device with cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) double2 g_noalloc_scratch[kMaxElems + 16];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (set-up on the
// first call per device, with that device current).
cudaError_t scratch_on_current_device(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

struct Geo { int L[4], b[4], c[4], bvol, V; };

// storage site s (aggregate-major, lexicographic inside the aggregate) -> lexicographic site
__device__ __forceinline__ int lex_of_storage(const Geo& g, int s) {
  int blk = s / g.bvol, loc = s % g.bvol;
  int x[4];
  for (int k = 0; k < 4; ++k) {
    const int xc = blk % g.c[k];
    blk /= g.c[k];
    const int xl = loc % g.b[k];
    loc /= g.b[k];
    x[k] = xc * g.b[k] + xl;
  }
  return x[0] + g.L[0] * (x[1] + g.L[1] * (x[2] + g.L[2] * x[3]));
}

__global__ void k_na_pack(double2* __restrict__ dst, const double2* __restrict__ ext, Geo g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (s >= g.V) return;
  const double2* e = ext + ((long long)i * g.V + lex_of_storage(g, s)) * 12;
  double2* d = dst + (long long)i * 12 * g.V;
  for (int c = 0; c < 12; ++c) d[(long long)c * g.V + s] = e[c];
}

__global__ void k_na_unpack(double2* __restrict__ ext, const double2* __restrict__ src, Geo g) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (s >= g.V) return;
  double2* e = ext + ((long long)i * g.V + lex_of_storage(g, s)) * 12;
  const double2* d = src + (long long)i * 12 * g.V;
  for (int c = 0; c < 12; ++c) e[c] = d[(long long)c * g.V + s];
}

}  // namespace
}  // namespace wcmg

extern "C" int wcmg_block_orthonormalise_noalloc(const void* vecs_in, void* vecs_out, const int dims[4],
                                                 const int block[4], int nvec, void* stream) {
  using namespace wcmg;
  if (!vecs_in || !vecs_out || !dims || !block) return WCMG_ERR_ARG;
  Geo g;
  long long V = 1;
  g.bvol = 1;
  for (int k = 0; k < 4; ++k) {
    if (dims[k] < 1 || block[k] < 1 || dims[k] % block[k]) return WCMG_ERR_ARG;
    g.L[k] = dims[k];
    g.b[k] = block[k];
    g.c[k] = dims[k] / block[k];
    V *= dims[k];
    g.bvol *= block[k];
  }
  if (nvec < 1 || nvec > 32 || g.bvol * 6 < nvec || g.bvol * 6 > 2048) return WCMG_ERR_ARG;
  if ((long long)nvec * V * 12 > kMaxElems) return WCMG_ERR_ARG;  // beyond the fixed scratch
  g.V = (int)V;
  double2* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) return WCMG_ERR_CUDA;
  int* err = reinterpret_cast<int*>(scratch + kMaxElems);
  cudaStream_t st = (cudaStream_t)stream;
  try {
    WCMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));  // the array keeps the last call's contents
    k_na_pack<<<dim3(nblk(V, 128), nvec), 128, 0, st>>>(scratch, (const double2*)vecs_in, g);
    WCMG_LAUNCH_CHECK();
    launch_block_ortho(scratch, g.V, 12, g.bvol, nvec, true, err, st);
    k_na_unpack<<<dim3(nblk(V, 128), nvec), 128, 0, st>>>((double2*)vecs_out, scratch, g);
    WCMG_LAUNCH_CHECK();
    int h_err = 0;
    WCMG_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    WCMG_CUDA(cudaStreamSynchronize(st));
    if (h_err) return WCMG_ERR_NAN;
  } catch (const Error& e) {
    return e.code;
  }
  return WCMG_OK;
}
