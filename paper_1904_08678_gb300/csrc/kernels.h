// Host-side launchers of the wcmg CUDA kernels (one declaration per kernel family).
#pragma once
#include "common.cuh"

namespace wcmg {

// Geometry of one level as seen by its stencil kernels.  Sites are stored in
// hierarchical block-major order: the |B| sites of one aggregate of the next
// coarser level are contiguous, so transfers need no index tables.
struct LevelGeom {
  int V;            // sites
  const int* nbr;   // [8][V] storage index of x + mu (2 mu) and x - mu (2 mu + 1)
  int b[4];         // aggregate extents towards the next level (1s on the coarsest)
  int bvol;         // b0 * b1 * b2 * b3
  const unsigned char* par = nullptr;  // [V] site parity (x + y + z + t) % 2 (ST_PARITY)
};

// ST_PARITY (coarse levels): the full nine-point stencil on the sites whose parity is
// `hopdir`, zero on the others (the even-odd Schur complement of the coarsest solve).
enum StencilMode { ST_FULL = 0, ST_BLOCK_INTERIOR = 1, ST_FACE_HOP = 2, ST_PARITY = 3 };

// one bounded mbarrier wait that nothing completes: sets *err = 3 (coarse.cu)
void launch_wait_selftest(int* err, long long polls, cudaStream_t st);

// ---- fine level (fine.cu) ----
template <typename R>
void launch_pack_fine(cplx<R>* out, const double2* ext, const int* perm, int V, int nrhs, cudaStream_t st);
template <typename R>
void launch_unpack_fine(double2* ext, const cplx<R>* in, const int* perm, int V, int nrhs, cudaStream_t st);
template <typename R>
void launch_pack_gauge(cplx<R>* out, const double2* ext, const int* perm, int V, cudaStream_t st);
void launch_clover_build(double2* clov, const double2* gauge64, const int* nbr, int V, double m0, double csw,
                         cudaStream_t st);
void launch_clover_expand(double2* ext, const double2* clov, const int* perm, int V, cudaStream_t st);
// External [V][12][12] site blocks -> packed clover layout; *bad (zeroed by the
// caller) becomes nonzero at a site whose block is not Hermitian and block diagonal
// in chirality to tol relative to the block's largest entry, or is not finite.
void launch_clover_pack(double2* clov, const double2* ext, const int* perm, int V, double tol, int* bad,
                        cudaStream_t st);
// colour non-null: only the sites of the aggregates B with colour[B] == col are computed
// and written (the SAP residual of one colour pass); the others keep `out`.
template <typename R>
void launch_dslash(cplx<R>* out, const cplx<R>* in, const cplx<R>* gauge, const cplx<R>* clov, const LevelGeom& g,
                   int nrhs, int mode, int hopdir, cudaStream_t st, const unsigned char* colour = nullptr,
                   int col = 0);
// One SAP colour pass on the fine level, fused: for each aggregate B in blocks[0 ..
// nblocks) and every rhs, r = b - Dx on B (Dx null: b), `steps` MR steps of the
// block-local D_B from e = 0 with alpha_B = <p, r>_B / <p, p>_B, then x += e on B.
// Aggregates of at most 256 sites (sap_fine_threads(bvol) != 0).
int sap_fine_threads(int bvol);
template <typename R>
void launch_sap_fine(cplx<R>* x, const cplx<R>* b, const cplx<R>* Dx, const cplx<R>* gauge, const cplx<R>* clov,
                     const LevelGeom& g, const int* blocks, int nblocks, int steps, int nrhs, cudaStream_t st);
// C(x)^-1 in the packed clover layout (FP64 Gauss-Jordan per site and chirality);
// err receives 1 on a singular site block.
void launch_clover_invert(double2* inv, const double2* clov, int V, int* err, cudaStream_t st);
// The same pass with even-odd preconditioned block solves: MR on each block's Schur
// complement on its odd sites (cinv = C^-1; opar[B] = parity of block B's first site).
// Aggregates of at most 256 sites with an even x extent.
template <typename R>
void launch_sap_fine_eo(cplx<R>* x, const cplx<R>* b, const cplx<R>* Dx, const cplx<R>* gauge, const cplx<R>* clov,
                        const cplx<R>* cinv, const LevelGeom& g, const int* blocks, const unsigned char* opar,
                        int nblocks, int steps, int nrhs, cudaStream_t st);
// out = D in (full stencil) and, per rhs r, pr[r] = <out_r, in_r> = sum conj(out) in,
// pp[r] = <out_r, out_r> (the minimal-residual step's two reductions, fused into the
// stencil).  pr_part / pp_part: scratch of nrhs * dslash_partials(V) entries.
int dslash_partials(int V);
// Masked stencil (ST_BLOCK_INTERIOR or ST_FACE_HOP) of both chirality projections of
// nv vectors: out[i] = D_mode(Pi_+ v_i), out[nv + i] = D_mode(Pi_- v_i) (CoarsenOperator).
template <typename R>
void launch_dslash_chiral(cplx<R>* out, const cplx<R>* vecs, const cplx<R>* gauge, const cplx<R>* clov,
                          const LevelGeom& g, int nv, int mode, int hopdir, cudaStream_t st);
template <typename R>
void launch_dslash_mr(cplx<R>* out, const cplx<R>* in, const cplx<R>* gauge, const cplx<R>* clov, const LevelGeom& g,
                      int nrhs, double2* pr, double* pp, double2* pr_part, double* pp_part, cudaStream_t st);

// ---- transfers (transfer.cu) ----
// `fine` selects the component-major fine layout [ncomp][V]; otherwise fields are
// site-major [V][ncomp].  Vectors and fields of one level share the layout.
// face >= 0 restricts only the sites on that face of every aggregate (2 mu: +mu
// face, 2 mu + 1: -mu face; `block` = aggregate extents); other sites are not read.
template <typename R>
void launch_restrict(cplx<R>* coarse, const cplx<R>* in, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                     int nrhs, bool fine, cudaStream_t st, int face = -1, const int* block = nullptr);
template <typename R>
void launch_prolong(cplx<R>* out, const cplx<R>* coarse, const cplx<R>* vecs, int Vf, int nc, int bvol, int nvec,
                    int nrhs, bool fine, cudaStream_t st);
// FP64 block orthonormalisation in place; err receives 1 on a rank-deficient panel.
void launch_block_ortho(double2* vecs, int Vf, int nc, int bvol, int nvec, bool fine, int* err, cudaStream_t st);
// The same in double-float arithmetic on the FP32 pipe (48-bit significands, FP64
// output in vecs); qdf: scratch of as many float4 as vecs has complex entries.  The
// input is vecs itself, or the FP32 field in32 when given; out32 (nullable) receives
// the FP32 rounding of the result as well.
void launch_block_ortho_df(double2* vecs, float4* qdf, int Vf, int nc, int bvol, int nvec, bool fine, int* err,
                           cudaStream_t st, const float2* in32 = nullptr, float2* out32 = nullptr);
// cols[b] = Pi_s v_i with (s, i) = divmod(b0 + b, nvec), for b < ncols.
template <typename R>
void launch_make_columns(cplx<R>* cols, const cplx<R>* vecs, int Vf, int nc, int nvec, int b0, int ncols, bool fine,
                         cudaStream_t st);

// ---- coarse levels (coarse.cu) ----
// Even-odd coarsest solve: inv[x] = A_0(x)^-1 (row-major nb x nb, FP64) of every site by
// Gauss-Jordan with partial pivoting; *err = 1 on a singular block.
template <typename L>
void launch_self_invert(double2* inv, const L* links, int Vc, int nb, int* err, cudaStream_t st);
// out[x] = inv[x] in[x] on the sites of parity p, 0 elsewhere (nrhs fields [nrhs][Vc][nb]).
template <typename R>
void launch_blockinv_apply(cplx<R>* out, const cplx<R>* in, const cplx<R>* inv, const unsigned char* par, int p,
                           int Vc, int nb, int nrhs, cudaStream_t st);
// out = a + beta b on the sites of parity p, 0 elsewhere.
template <typename R>
void launch_parity_axpy(cplx<R>* out, const cplx<R>* a, const cplx<R>* b, double beta, const unsigned char* par, int p,
                        int Vc, int nb, int nrhs, cudaStream_t st);
// Coarse links: per site a row-major nb x ld matrix, ld = round_up(9 nb, 4),
// column d*nb + c of row a holds A_d(x)[a][c].
inline int links_ld(int nb) { return (9 * nb + 3) / 4 * 4; }
// row stride of the five-block storage [A_0 | A_{+x} | A_{+y} | A_{+z} | A_{+t}] (kind 5)
inline int links5_ld(int nb) { return (5 * nb + 3) / 4 * 4; }
template <typename L>
void launch_pack_links(L* links, const double2* ext, const int* perm, int Vc, int nb, cudaStream_t st);
template <typename L>
void launch_unpack_links(double2* ext, const L* links, const int* perm, int Vc, int nb, cudaStream_t st);
template <typename R>
void launch_pack_coarse(cplx<R>* out, const double2* ext, const int* perm, int V, int nc, int nrhs, cudaStream_t st);
template <typename R>
void launch_unpack_coarse(double2* ext, const cplx<R>* in, const int* perm, int V, int nc, int nrhs, cudaStream_t st);
// Launch shape of the coarse apply.  kind 0: one-rhs kernel (parts CTAs per
// site, threads per CTA); kind 1: rhs-tile kernel (rr rhs per CTA, parts CTAs
// per site, 0 = automatic); kind 2: tcgen05 tensor-core kernel (BF16 links, N
// tile ntile).  kind -1: the fixed rule of coarse_default_tile.
// kind 3: one-rhs streaming pipeline (threads per CTA, parts = link rows per staged
// chunk, stages = chunks in flight); kind 4: tcgen05 multi-rhs apply fed by bulk copies
// (ntile rhs per N tile, threads = MMA M (64 or 128), stages); kind 5: one-rhs kernel on
// the five-block storage of a Galerkin operator (parts, threads, stages as kind 0).
struct CoarseTile {
  int kind = -1, rr = 0, parts = 0, threads = 0, ntile = 0, stages = 0;
};
// Shared memory of the one-rhs streaming kernel (kind 3).
size_t coarse_stream_smem(int nb, int cr, int stages, int vec_bytes, int link_bytes);
// link_kind: 0 FP64, 1 FP32, 2 BF16, 3 FP16 link storage
CoarseTile coarse_default_tile(int nb, int nrhs, int mode, int Vc, int link_kind);
bool coarse_tile_valid(const CoarseTile& t, int nb, int nrhs, int mode, int link_kind);
// err (device int, may be null): receives 3 if a bounded wait of the tensor-core
// path gave up; a null err keeps the SIMT kernels.  tile (nullable): launch shape
// (validated; an invalid tile throws).
// lmma / scratch: the MMA copy of BF16 links (launch_links_to_mma) and a scratch of at
// least coarse_mma4_scratch_bytes bytes, both needed by kind 4 (otherwise the fixed rule).
// links5: the five-block copy (launch_links_to_5), needed by kind 5 (otherwise the fixed
// rule); valid only for links with A_{-mu}(x) = sigma3 A_{+mu}(x - mu)^dag sigma3.
template <typename R, typename L>
void launch_coarse_apply(cplx<R>* out, const cplx<R>* in, const L* links, const LevelGeom& g, int nb, int nrhs,
                         int mode, int hopdir, cudaStream_t st, int* err = nullptr,
                         const CoarseTile* tile = nullptr, const bf16c* lmma = nullptr, void* scratch = nullptr,
                         size_t scratch_bytes = 0, const L* links5 = nullptr);
// kind 5: the five-block copy (self + forward hops) of a Galerkin operator's links
template <typename L>
void launch_links_to_5(L* dst, const L* src, int Vc, int nb, cudaStream_t st);
// kind 4 (tcgen05 fed by bulk copies): the links in the MMA's K-major core-matrix order,
// [site][d][16-byte group g][row a]; its shared memory; its scratch for any rhs tile.
void launch_links_to_mma(bf16c* dst, const bf16c* src, int Vc, int nb, cudaStream_t st);
size_t coarse_mma4_smem(int nb, int ntile, int mm, int stages);
size_t coarse_mma4_scratch_bytes(int Vc, int nb, int nrhs);
// links[x][a][d*nb + b0 + j] = res[j][x][a] for j < ncols (res: restrict output of the column fields)
template <typename R, typename L>
void launch_scatter_links(L* links, const cplx<R>* res, int Vc, int nb, int d, int b0, int ncols, cudaStream_t st);
template <typename Lin, typename Lout>
void launch_convert_links(Lout* out, const Lin* in, long long n, cudaStream_t st);

// ---- BLAS-1 and Krylov helpers (blas.cu); fields are [nrhs][n] complex ----
template <typename A, typename B>
void launch_convert(cplx<B>* out, const cplx<A>* in, long long n, cudaStream_t st);
template <typename R>
void launch_dot(double2* out, const cplx<R>* a, const cplx<R>* b, long long n, int nrhs, double2* partial,
                cudaStream_t st);
template <typename R>
void launch_norm2(double* out, const cplx<R>* a, long long n, int nrhs, double* partial, cudaStream_t st);
// out[r][i] = <basis_i, w> for i < k; basis_i at basis + i * bstride (each [nrhs][n]).
// kdev (nullable, device): the count is *kdev + kadd instead (at most k, which sizes
// the grid) -- the Arnoldi step number of a device-driven loop.
template <typename R>
void launch_multidot(double2* out, const cplx<R>* basis, long long bstride, int k, int ldo, const cplx<R>* w,
                     long long n, int nrhs, double2* partial, cudaStream_t st, const int* kdev = nullptr,
                     int kadd = 0);
// w[r] += sign * sum_{i<k} coef[r*ldc + i] * basis_i[r]; kdev as for launch_multidot
template <typename R>
void launch_multiaxpy(cplx<R>* w, const cplx<R>* basis, long long bstride, int k, const double2* coef, int ldc,
                      double sign, long long n, int nrhs, cudaStream_t st, const int* kdev = nullptr, int kadd = 0);
// dst[o * dmul + i] = src[o * smul + i] for i < n, o = *idx (0 if idx is null)
template <typename R>
void launch_copy_idx(cplx<R>* dst, const cplx<R>* src, long long n, const int* idx, long long dmul, long long smul,
                     cudaStream_t st);
void launch_fill_int(int* x, int v, int n, cudaStream_t st);
template <typename R>
void launch_axpby(cplx<R>* y, double a, const cplx<R>* x, double b, long long n, int nrhs, cudaStream_t st);
// y[r] = x[r] * s[r] (s real, device; 1/sqrt(s) with inv_sqrt).  ydev (nullable):
// y is offset by (*ydev + yadd) * ystride on the device.
template <typename R>
void launch_scale_dev(cplx<R>* y, const cplx<R>* x, const double* s, int inv_sqrt, long long n, int nrhs,
                      cudaStream_t st, const int* ydev = nullptr, int yadd = 0, long long ystride = 0);
// MR update with alpha[r] = pr[r] / pp[r] (0 if pp = 0), pr = <p, r>, pp = <p, p>:
//   x += alpha r ; r -= alpha p
// x_zero: x is taken as 0 and not read; r_next = false: r is not written (the last step
// of a fixed-step MR, whose residual nobody reads); rin (nullable): read the residual
// from rin instead of r (the first step reads b) and write the new one to r.
template <typename R>
void launch_mr_update(cplx<R>* x, cplx<R>* r, const cplx<R>* p, const double2* pr, const double* pp, long long n,
                      int nrhs, cudaStream_t st, bool x_zero = false, bool r_next = true,
                      const cplx<R>* rin = nullptr);
// x[r] = mask[r] ? 0 : x[r]
template <typename R>
void launch_mask_rhs(cplx<R>* x, const int* mask, long long n, int nrhs, cudaStream_t st);
template <typename R>
void launch_fill_zero(cplx<R>* x, long long n, cudaStream_t st);
// nfields complex Gaussian fields of n entries, field i from the counter-based generator
// with stream stream0 + i (SplitMix64 finaliser + Box-Muller, the seeded-input scheme)
void launch_counter_gaussian(double2* out, long long n, int nfields, unsigned long long seed,
                             unsigned long long stream0, cudaStream_t st);

// ---- SAP smoother (sap.cu) ----
// Blocks are the level's aggregates (block B = sites [B bvol, (B+1) bvol)); colour[B]
// is 0 or 1.  fine: fields component-major [nc][V], else site-major [V][nc].
// r = colour == c ? b - Dx : 0 per element (Dx null: b - 0)
template <typename R>
void launch_sap_residual(cplx<R>* r, const cplx<R>* b, const cplx<R>* Dx, const unsigned char* colour, int c, int V,
                         int nc, int bvol, bool fine, int nrhs, cudaStream_t st);
// One block-local MR step on the blocks of colour c (p = D_B r):
//   alpha_B = <p, r>_B / <p, p>_B (0 if <p, p>_B = 0); x += alpha_B r; r -= alpha_B p
template <typename R>
void launch_sap_block_mr(cplx<R>* x, cplx<R>* r, const cplx<R>* p, const unsigned char* colour, int c, int V, int nc,
                         int bvol, bool fine, int nrhs, cudaStream_t st);

// Arnoldi/Givens bookkeeping for batched (F)GMRES, one thread per rhs.
struct GmresState {
  double2* H;      // [nrhs][m+1][m]
  double* cs;      // [nrhs][m]
  double2* sn;     // [nrhs][m]
  double2* g;      // [nrhs][m+1]
  double2* y;      // [nrhs][m]
  double* hnorm;   // [nrhs]
  double* bnorm;   // [nrhs]
  double* resid;   // [nrhs]  |g_{j+1}|
  int* active;     // [nrhs]  1 while iterating in this cycle
  int* jdone;      // [nrhs]  steps taken in this cycle
  int* done;       // [nrhs]  finished for good (frozen in later cycles)
  int m;
};
// h column j is in H (entries 0..j from multidot); hnorm holds ||w||.
// h1, h2: the two CGS passes' coefficients [nrhs][m+1]; hnorm2 = ||w||^2 after both.
// `final_done`: a recurrence convergence also marks the rhs done (no true-residual check).
// One fused Arnoldi step after the operator application, for one short rhs
// (n <= 2^17, restart <= 64): CGS2 projections of w against V_0..V_j, the norm,
// the Givens update of Hessenberg column j and V_{j+1} = w / ||w||, in one launch
// of a thread-block cluster (16 CTAs, else 8).  jdev (nullable): step on the device.
bool arnoldi_fused_ok(long long n, int nrhs, int m);
template <typename R>
void launch_arnoldi_fused(cplx<R>* Vb, long long bstride, cplx<R>* w, long long n, const GmresState& S, int j,
                          const int* jdev, double tol, int final_done, cudaStream_t st);
// jdev (nullable, device): the step number is *jdev instead of j.
void launch_gmres_step(const GmresState& s, int j, const double2* h1, const double2* h2, const double* hnorm2,
                       double tol, int final_done, int nrhs, double* inv_h, cudaStream_t st,
                       const int* jdev = nullptr);
// done[r] |= nrm2[r] <= (tol * bnorm[r])^2
void launch_gmres_mark_done(const GmresState& s, const double* nrm2, double tol, int nrhs, cudaStream_t st);
void launch_gmres_solve_y(const GmresState& s, int nrhs, cudaStream_t st);
// start a cycle: beta[r] = sqrt(nrm2[r]); g = (beta, 0...); active = beta > tol*bnorm; inv_beta
void launch_gmres_start(const GmresState& s, const double* nrm2, double tol, int nrhs, double* inv_beta,
                        cudaStream_t st);

}  // namespace wcmg

namespace wcmg {
void launch_sqrt_inplace(double* x, int n, cudaStream_t st);
}

namespace wcmg {
// ---- learned coarse correction: PTC network (ptc.cu), FP32 fields [12][V] ----
void launch_ptc_forward(float2* out, const float2* in, const float2* W, const float2* U, const int* nbr, int V,
                        int nin, int nout, int nrhs, cudaStream_t st);
void launch_ptc_backward_data(float2* gin, const float2* gout, const float2* W, const float2* U, const int* nbr, int V,
                              int nin, int nout, int nrhs, cudaStream_t st);
long long ptc_wgrad_partial_size(int V, int nin, int nout, int nrhs);
void launch_ptc_wgrad(float2* gW, float2* partial, const float2* gout, const float2* in, const float2* U,
                      const int* nbr, int V, int nin, int nout, int nrhs, cudaStream_t st);
void launch_ptc_adam(float2* w, const float2* g, float2* m, float2* v, int n, float lr, int t, cudaStream_t st);
void launch_gaussian_field(float2* out, long long n, unsigned long long seed, unsigned long long stream,
                           cudaStream_t st);
}  // namespace wcmg

namespace wcmg {
// ---- device-driven Krylov loops (graph.cu) ----
// The stopping tests of (F)GMRES run on the device so that a whole solve can be
// captured once as a CUDA graph: each loop is a conditional WHILE node whose
// body ends with one of these single-block control kernels; the kernel updates
// the counters and sets the node's condition.  Every loop counter only grows and
// is capped (maxiter, restart length, KCTL_HARD_CAP), so each loop terminates.
constexpr int KCTL_HARD_CAP = 100000;
struct KCtl {
  int j;        // Arnoldi step within the current cycle
  int its;      // iterations of this invocation
  int cycles;   // restart cycles
  int stop;     // set once the invocation is finished
  int err;      // 1: non-finite residual norm
  int maxiter;  // iteration budget of this invocation
  int restarts; // (outer defect-correction loop) restarts
  int pad;
};
// Launch-count bookkeeping of graph replays: after a body executes, its control
// kernel adds body_counts[slot] (the number of kernels captured directly in
// that body, written by the host after capture) to *launches.
struct BodyCount {
  const int* counts;
  int slot;          // -1: do not count
  long long* launches;
};
// ctl: j = its = cycles = stop = err = restarts = 0; maxiter = budget_its ?
// min(maxiter, budget_max - *budget_its) : maxiter; if use_h, condition(h) = maxiter > 0.
void launch_kctl_init(KCtl* k, int maxiter, const int* budget_its, int budget_max,
                      cudaGraphConditionalHandle h, int use_h, cudaStream_t st);
// start of a cycle: j = 0; condition(h) = any(active) && m > 0 && its < maxiter
void launch_kctl_cycle_begin(KCtl* k, const int* active, int nrhs, int m, cudaGraphConditionalHandle h,
                             cudaStream_t st);
// end of an Arnoldi step: j++, its++, (*acc)++ if acc;
// condition(h) = any(active) && j < m && its < maxiter
void launch_kctl_step_end(KCtl* k, const int* active, int nrhs, int m, long long* acc, BodyCount bc,
                          cudaGraphConditionalHandle h, cudaStream_t st);
// end of a cycle: cycles++; stop = (max_cycles > 0 && cycles >= max_cycles) ||
// (!verify && all(done)) || cycles >= KCTL_HARD_CAP; condition(h_if) = !stop
// (h_if guards the true-residual step of the restart)
void launch_kctl_cycle_end(KCtl* k, const int* done, int nrhs, int verify, int max_cycles, BodyCount bc,
                           cudaGraphConditionalHandle h_if, cudaStream_t st);
// after the IF node of a restart: if the true-residual step ran (stop == 0), count
// its body, err/stop on a non-finite norm, stop when all(done), its >= maxiter or
// the cycle took no step; condition(h_loop) = !stop
void launch_kctl_restart_check(KCtl* k, const int* done, const double* nrm2, int nrhs, BodyCount bc_if,
                               cudaGraphConditionalHandle h_loop, cudaStream_t st);
// Defect-correction loop of the mixed-precision solve.  inner (nullable) is the
// FP32 FGMRES just run: its += inner->its, restarts++, and no progress
// (inner->its == 0) stops.  done[q] = ||r_q|| <= tol ||b_q|| (nrm2, bn2 squared
// norms); *worst = max_q ||r_q|| / ||b_q||; condition(h) = !all(done) && its <
// maxiter && !err.
void launch_mx_check(KCtl* k, const KCtl* inner, const double* nrm2, const double* bn2, double tol, int* done,
                     double* worst, int nrhs, BodyCount bc, cudaGraphConditionalHandle h, cudaStream_t st);
}  // namespace wcmg
