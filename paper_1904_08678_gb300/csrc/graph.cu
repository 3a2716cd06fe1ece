// Control kernels of the device-driven (F)GMRES loops (Sec. 2.1 solvers): the
// loop decisions that the host-driven solver takes after reading flags back are
// taken here on the device, so a whole solve runs as one CUDA graph with
// conditional WHILE / IF nodes and no host round trip.  Each kernel is one block;
// thread 0 updates the counters and sets the graph condition.
#include "kernels.h"

namespace wcmg {

constexpr int CTL_T = 128;

__device__ __forceinline__ int block_any(const int* f, int n) {
  int v = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) v |= f[r] != 0;
  return __syncthreads_or(v);
}
__device__ __forceinline__ int block_all(const int* f, int n) {
  int v = 1;
  for (int r = threadIdx.x; r < n; r += blockDim.x) v &= f[r] != 0;
  return __syncthreads_and(v);
}
__device__ __forceinline__ void count_body(const BodyCount& bc) {
  if (bc.launches && bc.slot >= 0) *bc.launches += bc.counts[bc.slot];
}

__global__ void k_kctl_init(KCtl* k, int maxiter, const int* budget_its, int budget_max,
                            cudaGraphConditionalHandle h, int use_h) {
  if (threadIdx.x != 0) return;
  int mi = maxiter;
  if (budget_its) mi = min(mi, budget_max - *budget_its);
  if (mi < 0) mi = 0;
  k->j = 0; k->its = 0; k->cycles = 0; k->stop = 0; k->err = 0; k->restarts = 0;
  k->maxiter = mi;
  if (use_h) cudaGraphSetConditional(h, mi > 0 ? 1u : 0u);
}

__global__ void k_kctl_cycle_begin(KCtl* k, const int* active, int nrhs, int m, cudaGraphConditionalHandle h) {
  const int any = block_any(active, nrhs);
  if (threadIdx.x != 0) return;
  k->j = 0;
  const int go = any && m > 0 && k->its < k->maxiter && k->its < KCTL_HARD_CAP;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_kctl_step_end(KCtl* k, const int* active, int nrhs, int m, long long* acc, BodyCount bc,
                                cudaGraphConditionalHandle h) {
  const int any = block_any(active, nrhs);
  if (threadIdx.x != 0) return;
  const int j = k->j + 1, its = k->its + 1;
  k->j = j;
  k->its = its;
  if (acc) *acc += 1;
  count_body(bc);
  const int go = any && j < m && its < k->maxiter && its < KCTL_HARD_CAP;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_kctl_cycle_end(KCtl* k, const int* done, int nrhs, int verify, int max_cycles, BodyCount bc,
                                 cudaGraphConditionalHandle h_if) {
  const int all = block_all(done, nrhs);
  if (threadIdx.x != 0) return;
  const int cyc = k->cycles + 1;
  k->cycles = cyc;
  const int stop = (max_cycles > 0 && cyc >= max_cycles) || (!verify && all) || cyc >= KCTL_HARD_CAP;
  k->stop = stop;
  count_body(bc);
  cudaGraphSetConditional(h_if, stop ? 0u : 1u);
}

// Runs after the IF node, directly in the restart loop's body, so that only
// kernels of the loop body itself set the loop's condition.
__global__ void k_kctl_restart_check(KCtl* k, const int* done, const double* nrm2, int nrhs, BodyCount bc_if,
                                     cudaGraphConditionalHandle h_loop) {
  int bad = 0;
  for (int r = threadIdx.x; r < nrhs; r += blockDim.x) bad |= !isfinite(nrm2[r]);
  bad = __syncthreads_or(bad);
  const int all = block_all(done, nrhs);
  if (threadIdx.x != 0) return;
  int stop = k->stop;
  if (!stop) {  // the true-residual body ran
    count_body(bc_if);
    if (bad) { k->err = 1; stop = 1; }
    if (all || k->its >= k->maxiter || k->j == 0) stop = 1;
  }
  k->stop = stop;
  cudaGraphSetConditional(h_loop, stop ? 0u : 1u);
}

__global__ void k_mx_check(KCtl* k, const KCtl* inner, const double* nrm2, const double* bn2, double tol, int* done,
                           double* worst, int nrhs, BodyCount bc, cudaGraphConditionalHandle h) {
  __shared__ double wmax[CTL_T];
  double w = 0.0;
  int bad = 0, all = 1;
  for (int q = threadIdx.x; q < nrhs; q += blockDim.x) {
    const double rn = nrm2[q], bn = bn2[q];
    bad |= !isfinite(rn);
    const double rel = bn > 0.0 ? sqrt(rn / bn) : 0.0;
    w = fmax(w, rel);
    const int d = rel <= tol;
    done[q] = d;
    all &= d;
  }
  wmax[threadIdx.x] = w;
  bad = __syncthreads_or(bad);
  all = __syncthreads_and(all);
  if (threadIdx.x != 0) return;
  for (int t = 1; t < blockDim.x; ++t) w = fmax(w, wmax[t]);
  *worst = w;
  int stalled = 0;
  if (inner) {
    k->its += inner->its;
    k->restarts += 1;
    stalled = inner->its == 0;
  }
  if (bad) k->err = 1;
  count_body(bc);
  const int go = !all && !bad && !stalled && k->its < k->maxiter && k->restarts < KCTL_HARD_CAP;
  k->stop = !go;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}

void launch_kctl_init(KCtl* k, int maxiter, const int* budget_its, int budget_max, cudaGraphConditionalHandle h,
                      int use_h, cudaStream_t st) {
  k_kctl_init<<<1, 32, 0, st>>>(k, maxiter, budget_its, budget_max, h, use_h);
  WCMG_LAUNCH_CHECK();
}
void launch_kctl_cycle_begin(KCtl* k, const int* active, int nrhs, int m, cudaGraphConditionalHandle h,
                             cudaStream_t st) {
  k_kctl_cycle_begin<<<1, CTL_T, 0, st>>>(k, active, nrhs, m, h);
  WCMG_LAUNCH_CHECK();
}
void launch_kctl_step_end(KCtl* k, const int* active, int nrhs, int m, long long* acc, BodyCount bc,
                          cudaGraphConditionalHandle h, cudaStream_t st) {
  k_kctl_step_end<<<1, CTL_T, 0, st>>>(k, active, nrhs, m, acc, bc, h);
  WCMG_LAUNCH_CHECK();
}
void launch_kctl_cycle_end(KCtl* k, const int* done, int nrhs, int verify, int max_cycles, BodyCount bc,
                           cudaGraphConditionalHandle h_if, cudaStream_t st) {
  k_kctl_cycle_end<<<1, CTL_T, 0, st>>>(k, done, nrhs, verify, max_cycles, bc, h_if);
  WCMG_LAUNCH_CHECK();
}
void launch_kctl_restart_check(KCtl* k, const int* done, const double* nrm2, int nrhs, BodyCount bc_if,
                               cudaGraphConditionalHandle h_loop, cudaStream_t st) {
  k_kctl_restart_check<<<1, CTL_T, 0, st>>>(k, done, nrm2, nrhs, bc_if, h_loop);
  WCMG_LAUNCH_CHECK();
}
void launch_mx_check(KCtl* k, const KCtl* inner, const double* nrm2, const double* bn2, double tol, int* done,
                     double* worst, int nrhs, BodyCount bc, cudaGraphConditionalHandle h, cudaStream_t st) {
  k_mx_check<<<1, CTL_T, 0, st>>>(k, inner, nrm2, bn2, tol, done, worst, nrhs, bc, h);
  WCMG_LAUNCH_CHECK();
}

}  // namespace wcmg
