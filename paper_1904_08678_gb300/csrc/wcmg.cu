// Host orchestration and C-ABI of the multigrid library (include/wcmg.h).
//
// Sec. 2.1 of the paper: the solver class calls itself recursively over the
// levels; the coarse operator of each level is applied through Mdiag + Mdir
// and can be coarsened again; MR is the smoother, GMRES the coarsest solver,
// FGMRES the outer solver; the setup is the smoother-based initial setup
// followed by iterative refinement with the whole MG preconditioner.  The
// precision change of the paper (double outer solver, single preconditioner) is
// the inner_prec = F32 mode, here with FP64 defect correction at every restart.
//
// Every Krylov loop is batched over right-hand sides: the setup runs all Nvec
// near-null candidates of a level as one batch, and each rhs keeps its own
// Hessenberg matrix and stopping state on the device.
#include "../../include/wcmg.h"
#include "kernels.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace wcmg {

// Bumped by every device allocation of a DevBuf and by every change of a coarse
// launch tile: a captured CUDA graph is valid only while no buffer it references
// has been reallocated and every launch shape it baked in still holds.
static unsigned long long& graph_epoch() {
  static unsigned long long g = 0;
  return g;
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  T* ensure(size_t count) {
    if (count <= n && p) return p;
    release();
    WCMG_CUDA(cudaMalloc(&p, (count ? count : 1) * sizeof(T)));
    n = count;
    ++graph_epoch();
    return p;
  }
};

struct HostGeom {
  int dims[4] = {1, 1, 1, 1};
  int V = 1;
  int b[4] = {1, 1, 1, 1};
  int bvol = 1;
  std::vector<int> perm, inv, nbr;
  DevBuf<int> d_perm, d_nbr;
  DevBuf<unsigned char> d_par;  // site parity (x + y + z + t) % 2 in storage order
  LevelGeom lg() const {
    LevelGeom g;
    g.V = V;
    g.nbr = d_nbr.p;
    g.par = d_par.p;
    for (int k = 0; k < 4; ++k) g.b[k] = b[k];
    g.bvol = bvol;
    return g;
  }
};

static inline int lexi(const int* x, const int* d) { return x[0] + d[0] * (x[1] + d[1] * (x[2] + d[2] * x[3])); }
static inline void coords(int s, const int* d, int* x) {
  x[0] = s % d[0]; s /= d[0];
  x[1] = s % d[1]; s /= d[1];
  x[2] = s % d[2];
  x[3] = s / d[2];
}

// Scalars of one level's Krylov loops (device) and its (F)GMRES state.
struct LevelScalars {
  int cap_rhs = 0, cap_m = 0;
  DevBuf<double2> c2;  // h1, h2 [2][rhs][m+1]; pr [rhs]
  DevBuf<double> d;    // hn2, nrm2, inv_beta, inv_h, pp, bnorm, resid, cs... [slots][rhs]
  DevBuf<double2> H, sn, g, y;
  DevBuf<double> cs;
  DevBuf<int> ints;    // active, jdone, done
  void ensure(int rhs, int m) {
    if (rhs <= cap_rhs && m <= cap_m) return;
    rhs = std::max(rhs, cap_rhs);
    m = std::max(m, cap_m);
    c2.ensure((size_t)rhs * (2 * (m + 1) + 1));
    d.ensure((size_t)rhs * 8);
    H.ensure((size_t)rhs * (m + 1) * m);
    sn.ensure((size_t)rhs * m);
    g.ensure((size_t)rhs * (m + 1));
    y.ensure((size_t)rhs * m);
    cs.ensure((size_t)rhs * m);
    ints.ensure((size_t)rhs * 3);
    cap_rhs = rhs;
    cap_m = m;
  }
  // a host-side check: every accessor needs the buffers (never hand a kernel a null pointer)
  void need() const {
    if (!c2.p || !d.p || !H.p || !ints.p) throw Error(WCMG_ERR_STATE, "Krylov scalars used before allocation");
  }
  double2* h1() { need(); return c2.p; }
  double2* h2() { need(); return c2.p + (size_t)cap_rhs * (cap_m + 1); }
  double2* pr() { need(); return c2.p + (size_t)2 * cap_rhs * (cap_m + 1); }
  double* slot(int k) { need(); return d.p + (size_t)k * cap_rhs; }
  GmresState state(int m) {
    need();
    if (m > cap_m) throw Error(WCMG_ERR_STATE, "Krylov scalars too small for the restart length");
    GmresState s;
    s.H = H.p; s.cs = cs.p; s.sn = sn.p; s.g = g.p; s.y = y.p;
    s.hnorm = slot(0); s.bnorm = slot(5); s.resid = slot(6);
    s.active = ints.p; s.jdone = ints.p + cap_rhs; s.done = ints.p + 2 * cap_rhs;
    s.m = m;
    return s;
  }
};
// slot map: 0 hn2, 1 nrm2, 2 inv_beta, 3 inv_h, 4 pp, 5 bnorm, 6 resid, 7 misc

struct Level {
  HostGeom g;
  int nc = 12;
  bool fine = true;
  int nvec = 0;  // towards the next level
  DevBuf<double2> v64;
  DevBuf<float2> v32;
  bool have_P = false, v32_valid = false;
  DevBuf<double2> raw64, raw64b;  // raw near-null vectors; b: the next sweep's output
  DevBuf<float2> raw32, raw32b;
  // coarse operator of this level (level >= 1)
  bool have_op = false;
  bool op64 = false;  // FP64 links present (else FP32)
  DevBuf<double2> L64;
  DevBuf<float2> L32;
  DevBuf<bf16c> Lbf;
  DevBuf<bf16c> Lmma;  // BF16 links in the tcgen05 operand order (kind-4 coarse apply)
  bool mma_valid = false;
  DevBuf<double2> Ainv64;  // even-odd coarsest solve: A_0(x)^-1 per site (FP64, FP32 copy)
  DevBuf<float2> Ainv32;
  bool ainv_valid = false;
  DevBuf<f16c> Lh;
  bool L32_valid = false, low_valid = false;
  // five-block copies per link kind (FP64, FP32, BF16, FP16) of a Galerkin operator
  // (sigma3: the links come from the setup's P^dag D P, so the hop blocks obey
  // A_{-mu}(x) = sigma3 A_{+mu}(x - mu)^dag sigma3)
  DevBuf<unsigned char> L5[4];
  bool l5_valid[4] = {false, false, false, false};
  bool sigma3 = false;
  LevelScalars sc;
  LevelScalars sc_s;  // the GMRES smoother's own Krylov state (it runs inside the outer FGMRES)
  DevBuf<unsigned char> colour;  // SAP: colour (coarse-coordinate parity) of each aggregate
  DevBuf<int> sap_list;          // SAP: the aggregates of colour 0, then those of colour 1
  DevBuf<unsigned char> opar;    // SAP: parity of each aggregate's first site (even-odd block solves)
  int sap_count[2] = {0, 0};
  std::map<std::string, DevBuf<unsigned char>> ws;
  // coarse-apply launch shape per (nrhs, link storage): tuned or forced
  struct TileInfo {
    CoarseTile t;
    int source = 0;  // 1 autotuned, 2 set by the caller
    int candidates = 0;
    double us = 0.0, us_default = 0.0;
  };
  std::map<std::pair<int, int>, TileInfo> tiles;
  long long n() const { return (long long)g.V * nc; }
};

struct Prof {
  int mask = 0;
  std::vector<cudaEvent_t> pool;
  struct Pend { int cls; cudaEvent_t a, b; double bytes, flops; };
  std::vector<Pend> pend;
  wcmg_kstat k[WCMG_NKCLASS];
  Prof() { reset(); }
  void reset() { std::memset(k, 0, sizeof(k)); }
  cudaEvent_t get() {
    if (pool.empty()) {
      cudaEvent_t e;
      WCMG_CUDA(cudaEventCreate(&e));
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  void flush() {
    for (auto& p : pend) {
      WCMG_CUDA(cudaEventSynchronize(p.b));
      float ms = 0;
      WCMG_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
      k[p.cls].ms += ms;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pend.clear();
  }
  ~Prof() {
    for (auto& p : pend) { pool.push_back(p.a); pool.push_back(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

}  // namespace wcmg

using namespace wcmg;

struct wcmg_ctx {
  wcmg_params p;
  std::string err;
  std::vector<Level> L;
  DevBuf<double2> gauge64, clover64, cinv64;  // cinv: C(x)^-1 (even-odd SAP), same packing as C
  DevBuf<float2> gauge32, clover32, cinv32;
  DevBuf<int> cinv_err;
  bool have_gauge = false;
  DevBuf<double2> partial;
  DevBuf<double> partial_d;
  DevBuf<unsigned char> l2flush;  // scratch written to evict L2 (cold autotuning)
  DevBuf<double2> mr_pr;   // per-CTA partials of the fused MR Dslash
  DevBuf<double> mr_pp;
  DevBuf<unsigned char> stage[3];
  DevBuf<int> errflag;
  DevBuf<int> tma_err;       // nonzero after a bounded device-side wait gave up
  int* h_flags = nullptr;   // pinned host mirror of per-rhs flags
  double* h_vals = nullptr; // pinned host mirror of per-rhs values
  int hcap = 0;
  Prof prof;
  long long opc[WCMG_NOPC][WCMG_MAX_LEVELS] = {};  // operator applications (wcmg_get_opcounts)
  bool in_coarsen = false;                         // the coarsening's stencils and restrictions are its own
  bool eo_schur = false;                           // the coarsest GMRES is running on the Schur complement
  cudaStream_t st = nullptr;
  long long coarse_its = 0;
  // learned coarse correction (PTC network)
  DevBuf<float2> ptcW, ptcG, ptcM, ptcV, ptcPartial;
  DevBuf<double> ptcScale;
  DevBuf<float2> ds_r, ds_e;
  bool have_ptc = false;
  int ptc_t = 0;
  int coarse_mode = WCMG_COARSE_MG;
  double fallback_ratio = 0.9;
  bool learned_on = false, learned_fallback = false;
  int learned_cycles = 0;
  // solve captured as one CUDA graph with device-side loop control
  static constexpr int MAX_CAP_DEPTH = 8, MAX_BODIES = 256;
  bool capturing = false;
  int cap_depth = 0;
  cudaStream_t cap_st[MAX_CAP_DEPTH] = {};
  std::vector<int> body_counts_h;         // kernels captured directly in each conditional body
  std::vector<long long> nested;          // capture-time stack: kernels of nested bodies
  DevBuf<int> body_counts;                // device copy of body_counts_h
  DevBuf<long long> gstat;                // [0] kernels launched by bodies, [1] coarsest GMRES iterations
  DevBuf<KCtl> kctl;                      // 0 mixed loop, 1 level-0 FGMRES, 2 + l coarsest GMRES,
                                          // 2 + WCMG_MAX_LEVELS + l GMRES smoother of level l
  DevBuf<int> mx_done;
  DevBuf<double> mx_worst;
  struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nrhs = 0;
    bool guess = false;                  // captured with the caller's initial guess (else x = 0)
    unsigned long long gen = 0;
    long long top_launches = 0;  // kernels outside conditional bodies
    void reset() {
      if (exec) cudaGraphExecDestroy(exec);
      if (g) cudaGraphDestroy(g);
      exec = nullptr;
      g = nullptr;
      nrhs = 0;
    }
  } graph;
  std::vector<int> warm_rhs;              // nrhs values already solved once (every workspace allocated)
  bool guess = false;                     // the solve being run or captured starts from the given x
  long long graph_top = 0;                // kernels of the last capture outside conditional bodies
  Graph batch;                            // wcmg_solve_batch graph (cached on the first context)
  std::vector<const void*> batch_key;
  ~wcmg_ctx() {
    graph.reset();
    batch.reset();
    for (auto s : cap_st)
      if (s) cudaStreamDestroy(s);
    if (h_flags) cudaFreeHost(h_flags);
    if (h_vals) cudaFreeHost(h_vals);
  }
};

namespace wcmg {

// Launch `call` (one kernel family of class `cls`); count it with its
// algorithmic bytes/flops and, when the class is in the profile mask, time it
// with a CUDA-event pair on the call's stream.
#define KPROF(c, cls, BYTES_, FLOPS_, call)                                        \
  do {                                                                           \
    const bool on_ = (((c)->prof.mask >> (cls)) & 1) && !(c)->capturing;        \
    cudaEvent_t a_ = nullptr, b_ = nullptr;                                      \
    if (on_) { a_ = (c)->prof.get(); WCMG_CUDA(cudaEventRecord(a_, (c)->st)); }  \
    call;                                                                        \
    (c)->prof.k[(cls)].launches += 1;                                            \
    (c)->prof.k[(cls)].bytes += (double)(BYTES_);                                \
    (c)->prof.k[(cls)].flops += (double)(FLOPS_);                                \
    if (on_) {                                                                   \
      b_ = (c)->prof.get();                                                      \
      WCMG_CUDA(cudaEventRecord(b_, (c)->st));                                   \
      (c)->prof.pend.push_back({(cls), a_, b_, 0.0, 0.0});                      \
    }                                                                            \
  } while (0)

static void host_mirrors(wcmg_ctx* c, int n) {
  if (n <= c->hcap) return;
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->h_vals) cudaFreeHost(c->h_vals);
  c->h_flags = nullptr;
  c->h_vals = nullptr;
  WCMG_CUDA(cudaMallocHost(&c->h_flags, sizeof(int) * n));
  WCMG_CUDA(cudaMallocHost(&c->h_vals, sizeof(double) * n));
  c->hcap = n;
}
static const int* read_ints(wcmg_ctx* c, const int* d, int n) {
  host_mirrors(c, n);
  WCMG_CUDA(cudaMemcpyAsync(c->h_flags, d, sizeof(int) * n, cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  return c->h_flags;
}
static const double* read_doubles(wcmg_ctx* c, const double* d, int n) {
  host_mirrors(c, n);
  WCMG_CUDA(cudaMemcpyAsync(c->h_vals, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  return c->h_vals;
}

template <typename R>
static cplx<R>* ws(Level& L, const char* name, long long nfields) {
  std::string key = std::string(name) + (sizeof(R) == 8 ? "/64" : "/32");
  auto& b = L.ws[key];
  return reinterpret_cast<cplx<R>*>(b.ensure((size_t)nfields * L.n() * sizeof(cplx<R>)));
}

static bool inner64(const wcmg_ctx* c) { return c->p.inner_prec == WCMG_F64; }

static int max_rhs_all(const wcmg_ctx* c) {
  int m = std::max(1, c->p.max_rhs);
  for (int l = 0; l + 1 < c->p.n_levels; ++l) m = std::max(m, c->p.nvec[l]);
  return m;
}
static void ensure_partials(wcmg_ctx* c) {
  const int r = std::max(max_rhs_all(c), 2 * c->p.nvec[0] + 1);
  const int k = std::max(c->p.outer_restart, c->p.coarse_restart) + 1 + 8;
  c->partial.ensure((size_t)r * k * 608);
  c->partial_d.ensure((size_t)r * 608);
}

// ---------------- accessors at a precision ----------------
template <typename R> struct Prec;
template <> struct Prec<double> {
  static double2* gauge(wcmg_ctx* c) { return c->gauge64.p; }
  static double2* clover(wcmg_ctx* c) { return c->clover64.p; }
  static double2* clover_inv(wcmg_ctx* c) { return c->cinv64.p; }
  static double2* vecs(wcmg_ctx*, Level& L) { return L.v64.p; }
  static DevBuf<double2>& raw(Level& L) { return L.raw64; }
  static DevBuf<double2>& raw_next(Level& L) { return L.raw64b; }
};
template <> struct Prec<float> {
  static float2* gauge(wcmg_ctx* c) { return c->gauge32.p; }
  static float2* clover(wcmg_ctx* c) { return c->clover32.p; }
  static float2* clover_inv(wcmg_ctx* c) { return c->cinv32.p; }
  static float2* vecs(wcmg_ctx* c, Level& L) {
    if (!L.v32_valid) {
      L.v32.ensure((size_t)L.nvec * L.n());
      launch_convert<double, float>(L.v32.p, L.v64.p, (long long)L.nvec * L.n(), c->st);
      L.v32_valid = true;
    }
    return L.v32.p;
  }
  static DevBuf<float2>& raw(Level& L) { return L.raw32; }
  static DevBuf<float2>& raw_next(Level& L) { return L.raw32b; }
};

static double sz(int prec) { return prec == WCMG_F64 ? 16.0 : prec == WCMG_F32 ? 8.0 : 4.0; }

// The kind-4 (tcgen05, bulk-copy) coarse apply reads the BF16 links in the MMA's
// operand order: refreshed with every new BF16 copy of a level's links.
static void build_mma_links(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  L.mma_valid = false;
  if (L.nc % 8 || L.nc > 64) return;
  L.Lmma.ensure((size_t)L.g.V * L.nc * 9 * L.nc);
  launch_links_to_mma(L.Lmma.p, L.Lbf.p, L.g.V, L.nc, c->st);
  L.mma_valid = true;
}

// Operands of the kind-4 apply for nrhs rhs at level l (BF16 links only): the MMA copy
// of the links and a workspace large enough for any rhs tile.
struct MmaOps {
  const bf16c* lmma = nullptr;
  void* scratch = nullptr;
  size_t bytes = 0;
};
static MmaOps mma_ops(wcmg_ctx* c, int l, int nrhs, int lk) {
  Level& L = c->L[l];
  MmaOps m;
  if (lk != 2 || nrhs < 2 || !L.mma_valid) return m;
  m.lmma = L.Lmma.p;
  m.scratch = ws<float>(L, "mma_b", nrhs + 63);
  m.bytes = coarse_mma4_scratch_bytes(L.g.V, L.nc, nrhs);
  return m;
}

// Five-block copies (kind 5) of the links present at level l, when params.coarse_sigma3
// is set and the level's operator is a Galerkin product.
template <typename Lt> struct LKind;
template <> struct LKind<double2> { static constexpr int v = 0; };
template <> struct LKind<float2> { static constexpr int v = 1; };
template <> struct LKind<bf16c> { static constexpr int v = 2; };
template <> struct LKind<f16c> { static constexpr int v = 3; };
template <typename Lt>
static void build_links5_of(wcmg_ctx* c, int l, const Lt* src) {
  Level& L = c->L[l];
  const int k = LKind<Lt>::v;
  L.L5[k].ensure((size_t)L.g.V * L.nc * links5_ld(L.nc) * sizeof(Lt));
  launch_links_to_5<Lt>(reinterpret_cast<Lt*>(L.L5[k].p), src, L.g.V, L.nc, c->st);
  L.l5_valid[k] = true;
}
static void build_links5(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  for (bool& v : L.l5_valid) v = false;
  if (!c->p.coarse_sigma3 || !L.sigma3 || !L.have_op) return;
  if (L.op64) build_links5_of<double2>(c, l, L.L64.p);
  if (L.L32_valid) build_links5_of<float2>(c, l, L.L32.p);
  if (L.low_valid && c->p.coarse_link_prec == WCMG_BF16) build_links5_of<bf16c>(c, l, L.Lbf.p);
  if (L.low_valid && c->p.coarse_link_prec == WCMG_F16) build_links5_of<f16c>(c, l, L.Lh.p);
}
template <typename Lt>
static const Lt* links5_of(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  const int k = LKind<Lt>::v;
  return c->p.coarse_sigma3 && L.sigma3 && L.l5_valid[k] ? reinterpret_cast<const Lt*>(L.L5[k].p) : nullptr;
}

// ---------------- coarse-apply autotuner ----------------
// Candidate launch shapes of the full nine-point coarse apply (K4 / K4m).
static std::vector<CoarseTile> coarse_candidates(int nb, int nrhs, int lk, bool have5) {
  std::vector<CoarseTile> v;
  auto add = [&](int kind, int rr, int parts, int threads, int ntile, int stages = 0) {
    CoarseTile t;
    t.kind = kind; t.rr = rr; t.parts = parts; t.threads = threads; t.ntile = ntile; t.stages = stages;
    if (coarse_tile_valid(t, nb, nrhs, ST_FULL, lk)) v.push_back(t);
  };
  if (nrhs == 1) {
    for (int th : {256, 512})
      for (int p : {1, 2, 4, 8})
        for (int rp : {1, 2}) add(0, 1, p, th, 0, rp);
    for (int p : {1, 2, 4, 8, 16}) add(1, 1, p, 0, 0);
    // five-block storage (Galerkin operators only)
    if (have5)
      for (int th : {128, 256, 512})
        for (int rp : {1, 2}) add(5, 1, 1, th, 0, rp);
    // streaming pipeline: chunks of 8 rows up to a whole site, 2 .. 6 in flight
    for (int cr : {8, 16, 24, nb})
      for (int stg : {2, 3, 4, 6}) add(3, 0, cr, 256, 0, stg);
    return v;
  }
  if (lk == 2) {  // tcgen05 fed by bulk copies: MMA M, rhs tile, pipeline depth
    const int full = std::min(64, (nrhs + 7) / 8 * 8);
    std::vector<int> nts;
    for (int nt : {16, 32, full})
      if (nt <= full && std::find(nts.begin(), nts.end(), nt) == nts.end()) nts.push_back(nt);
    for (int mm : {64, 128})
      for (int nt : nts)
        for (int stg : {3, 4, 6}) add(4, 0, 0, mm, nt, stg);
    // (one TMEM accumulator, parts 1, fits more CTAs per SM for the wide tiles but
    // serialises each tile's MMAs behind the previous tile's epilogue: slower on the
    // 48-rhs tiles measured, so it is no candidate; set_coarse_tile still takes it)
  }
  for (int rr : {1, 4, 8})
    if (rr <= nrhs || rr == 4)
      for (int p : {0, 1, 2, 4, 8, 16}) add(1, rr, p, 0, 0);
  if (lk == 2)
    for (int nt : {16, 32, 48, 64})
      if (nt <= (nrhs + 15) / 16 * 16) add(2, 0, 0, 0, nt);
  return v;
}

// Time every candidate on the level's own links (back-to-back applies, as in a
// Krylov loop) and keep the fastest; the fixed rule is timed too.
// cold: the links start in HBM for every timed apply (L2 overwritten by a 256 MiB
// scratch write before it; median of 9 single applies) -- the streaming case;
// otherwise 10 back-to-back applies, as inside a Krylov loop.
template <typename R, typename Lt>
static Level::TileInfo tune_coarse(wcmg_ctx* c, int l, const Lt* links, int nrhs, int lk, bool cold = false) {
  Level& L = c->L[l];
  const int nb = L.nc;
  cplx<R>* in = ws<R>(L, "tune_in", nrhs);
  cplx<R>* out = ws<R>(L, "tune_out", nrhs);
  launch_fill_zero<R>(in, L.n() * nrhs, c->st);
  const size_t flush_bytes = (size_t)256 << 20;
  if (cold) c->l2flush.ensure(flush_bytes);
  cudaEvent_t e0, e1;
  WCMG_CUDA(cudaEventCreate(&e0));
  WCMG_CUDA(cudaEventCreate(&e1));
  const int reps = 10;
  const MmaOps mo = mma_ops(c, l, nrhs, lk);
  const Lt* l5 = links5_of<Lt>(c, l);
  auto launch = [&](const CoarseTile* t) {
    launch_coarse_apply<R, Lt>(out, in, links, L.g.lg(), nb, nrhs, ST_FULL, 0, c->st, c->tma_err.p, t, mo.lmma,
                               mo.scratch, mo.bytes, l5);
  };
  auto time_one = [&](const CoarseTile* t) -> double {
    for (int i = 0; i < 2; ++i) launch(t);
    if (cold) {
      std::vector<float> ms(9);
      for (int i = 0; i < 9; ++i) {
        WCMG_CUDA(cudaMemsetAsync(c->l2flush.p, i & 0xFF, flush_bytes, c->st));
        WCMG_CUDA(cudaEventRecord(e0, c->st));
        launch(t);
        WCMG_CUDA(cudaEventRecord(e1, c->st));
        WCMG_CUDA(cudaEventSynchronize(e1));
        WCMG_CUDA(cudaEventElapsedTime(&ms[i], e0, e1));
      }
      std::sort(ms.begin(), ms.end());
      return 1e3 * ms[4];
    }
    WCMG_CUDA(cudaEventRecord(e0, c->st));
    for (int i = 0; i < reps; ++i) launch(t);
    WCMG_CUDA(cudaEventRecord(e1, c->st));
    WCMG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.0f;
    WCMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return 1e3 * ms / reps;
  };
  Level::TileInfo ti;
  ti.t = coarse_default_tile(nb, nrhs, ST_FULL, L.g.V, lk);
  try {
    ti.us_default = ti.us = time_one(nullptr);
    const auto cands = coarse_candidates(nb, nrhs, lk, l5 != nullptr);
    for (const auto& cand : cands) {
      const double us = time_one(&cand);
      if (us < ti.us) {
        ti.us = us;
        ti.t = cand;
      }
    }
    ti.candidates = (int)cands.size() + 1;
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ti.source = 1;
  return ti;
}

// Launch shape for the full coarse apply of level l with nrhs rhs: a tile set by
// the caller or found by the autotuner (params.autotune, tuned on first use and
// never while a graph is being captured); nullptr selects the fixed rule.
template <typename R, typename Lt>
static const CoarseTile* coarse_tile(wcmg_ctx* c, int l, const Lt* links, int nrhs, int lk) {
  Level& L = c->L[l];
  auto it = L.tiles.find({nrhs, lk});
  if (it != L.tiles.end()) return &it->second.t;
  if (!c->p.autotune || c->capturing) return nullptr;
  Level::TileInfo ti = tune_coarse<R, Lt>(c, l, links, nrhs, lk);
  ++graph_epoch();
  return &(L.tiles[{nrhs, lk}] = ti).t;
}

// ---------------- operators ----------------
template <typename R>
static void apply_op(wcmg_ctx* c, int l, cplx<R>* out, const cplx<R>* in, int nrhs, int mode = ST_FULL,
                     int hopdir = 0);

// Even-odd coarsest solve (Sec. 4 red-black preconditioning): the parity-restricted
// nine-point stencil, the self-block inverses and the odd-site Schur complement
//   S v = [D (v - A_ee^-1 [D v]_e)]_o   (v vanishing on the even sites)
// = A_oo v_o - A_oe A_ee^-1 A_eo v_o, zero on the even sites.
template <typename R>
static void apply_parity(wcmg_ctx* c, int l, cplx<R>* out, const cplx<R>* in, int nrhs, int parity) {
  apply_op<R>(c, l, out, in, nrhs, ST_PARITY, parity);
}
static void ensure_ainv(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  if (L.ainv_valid) return;
  if (c->capturing) throw Error(WCMG_ERR_STATE, "self-block inverses built inside a capture");
  const int nb = L.nc;
  L.Ainv64.ensure((size_t)L.g.V * nb * nb);
  L.Ainv32.ensure((size_t)L.g.V * nb * nb);
  WCMG_CUDA(cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->st));
  if (L.op64) launch_self_invert<double2>(L.Ainv64.p, L.L64.p, L.g.V, nb, c->errflag.p, c->st);
  else launch_self_invert<float2>(L.Ainv64.p, L.L32.p, L.g.V, nb, c->errflag.p, c->st);
  const int* e = read_ints(c, c->errflag.p, 1);
  if (e[0]) throw Error(WCMG_ERR_NAN, "singular coarse self block: no even-odd coarsest solve");
  launch_convert<double, float>(L.Ainv32.p, L.Ainv64.p, (long long)L.g.V * nb * nb, c->st);
  L.ainv_valid = true;
}
template <typename R> static const cplx<R>* ainv_of(Level& L);
template <> const double2* ainv_of<double>(Level& L) { return L.Ainv64.p; }
template <> const float2* ainv_of<float>(Level& L) { return L.Ainv32.p; }

template <typename R>
static void eo_schur_apply(wcmg_ctx* c, int l, cplx<R>* out, const cplx<R>* in, int nrhs) {
  Level& L = c->L[l];
  const int nb = L.nc;
  cplx<R>* t = ws<R>(L, "eo_t", nrhs);
  cplx<R>* z = ws<R>(L, "eo_z", nrhs);
  apply_parity<R>(c, l, t, in, nrhs, 0);  // [D v]_e
  KPROF(c, WCMG_K_COARSE, (double)L.g.V * nb * (nb + 2.0 * nrhs) * sizeof(cplx<R>), 8.0 * L.g.V / 2 * nb * nb * nrhs,
        launch_blockinv_apply<R>(z, t, ainv_of<R>(L), L.g.d_par.p, 0, L.g.V, nb, nrhs, c->st));
  launch_axpby<R>(z, 1.0, in, -1.0, L.n(), nrhs, c->st);  // v - A_ee^-1 [D v]_e
  apply_parity<R>(c, l, out, z, nrhs, 1);
}

template <typename R>
static void apply_op(wcmg_ctx* c, int l, cplx<R>* out, const cplx<R>* in, int nrhs, int mode, int hopdir) {
  Level& L = c->L[l];
  if (mode == ST_FULL && c->eo_schur && l == c->p.n_levels - 1) {
    eo_schur_apply<R>(c, l, out, in, nrhs);
    return;
  }
  if (mode == ST_FULL && !c->in_coarsen && !c->capturing) c->opc[WCMG_OPC_APPLY][l] += nrhs;
  if (l == 0) {
    if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
    const double V = L.g.V, s = sizeof(cplx<R>);
    const int cls = sizeof(R) == 8 ? WCMG_K_DSLASH64 : WCMG_K_DSLASH;
    KPROF(c, cls, V * s * (24.0 * nrhs + 72.0), V * 1872.0 * nrhs,
          launch_dslash<R>(out, in, Prec<R>::gauge(c), Prec<R>::clover(c), L.g.lg(), nrhs, mode, hopdir, c->st));
    return;
  }
  if (!L.have_op) throw Error(WCMG_ERR_STATE, "coarse operator of level not built");
  const int nb = L.nc;
  const double Vc = L.g.V, nb2 = (double)nb * nb;
  const double flops = Vc * 8.0 * 9.0 * nb2 * nrhs;
  if (sizeof(R) == 8) {
    if (!L.op64) throw Error(WCMG_ERR_ARG, "FP64 coarse apply needs FP64 links");
    const CoarseTile* t = mode == ST_FULL ? coarse_tile<double, double2>(c, l, L.L64.p, nrhs, 0) : nullptr;
    KPROF(c, WCMG_K_COARSE, Vc * (9.0 * nb2 * 16.0 + 2.0 * nb * 16.0 * nrhs), flops,
          (launch_coarse_apply<double, double2>((double2*)out, (const double2*)in, L.L64.p, L.g.lg(), nb, nrhs,
                                                mode, hopdir, c->st, c->tma_err.p, t, nullptr, nullptr, 0,
                                                links5_of<double2>(c, l))));
    return;
  }
  const int lp = c->p.coarse_link_prec;
  if (mode == ST_FULL && L.low_valid && (lp == WCMG_BF16 || lp == WCMG_F16)) {
    if (lp == WCMG_BF16) {
      const CoarseTile* t = coarse_tile<float, bf16c>(c, l, L.Lbf.p, nrhs, 2);
      const MmaOps mo = mma_ops(c, l, nrhs, 2);
      KPROF(c, WCMG_K_COARSE, Vc * (9.0 * nb2 * 4.0 + 2.0 * nb * 8.0 * nrhs), flops,
            (launch_coarse_apply<float, bf16c>((float2*)out, (const float2*)in, L.Lbf.p, L.g.lg(), nb, nrhs, mode,
                                               hopdir, c->st, c->tma_err.p, t, mo.lmma, mo.scratch, mo.bytes,
                                               links5_of<bf16c>(c, l))));
    } else {
      const CoarseTile* t = coarse_tile<float, f16c>(c, l, L.Lh.p, nrhs, 3);
      KPROF(c, WCMG_K_COARSE, Vc * (9.0 * nb2 * 4.0 + 2.0 * nb * 8.0 * nrhs), flops,
            (launch_coarse_apply<float, f16c>((float2*)out, (const float2*)in, L.Lh.p, L.g.lg(), nb, nrhs, mode,
                                              hopdir, c->st, c->tma_err.p, t, nullptr, nullptr, 0,
                                              links5_of<f16c>(c, l))));
    }
    return;
  }
  if (!L.L32_valid) {
    const long long n = (long long)L.g.V * nb * links_ld(nb);
    L.L32.ensure(n);
    launch_convert_links<double2, float2>(L.L32.p, L.L64.p, n, c->st);
    L.L32_valid = true;
    if (c->p.coarse_sigma3 && L.sigma3) build_links5_of<float2>(c, l, L.L32.p);
  }
  const CoarseTile* t = mode == ST_FULL ? coarse_tile<float, float2>(c, l, L.L32.p, nrhs, 1) : nullptr;
  KPROF(c, WCMG_K_COARSE, Vc * (9.0 * nb2 * 8.0 + 2.0 * nb * 8.0 * nrhs), flops,
        (launch_coarse_apply<float, float2>((float2*)out, (const float2*)in, L.L32.p, L.g.lg(), nb, nrhs, mode,
                                            hopdir, c->st, c->tma_err.p, t, nullptr, nullptr, 0,
                                            links5_of<float2>(c, l))));
}

template <typename R>
static void restrict_op(wcmg_ctx* c, int l, cplx<R>* coarse, const cplx<R>* fine, int nrhs, int face = -1) {
  Level& L = c->L[l];
  if (!L.have_P) throw Error(WCMG_ERR_STATE, "prolongator of level not built");
  if (!c->in_coarsen && !c->capturing) c->opc[WCMG_OPC_RESTRICT][l] += nrhs;
  const double s = sizeof(cplx<R>);
  const double frac = face < 0 ? 1.0 : 1.0 / L.g.b[face >> 1];  // share of the sites read
  KPROF(c, WCMG_K_RESTRICT,
        frac * (double)L.n() * s * (L.nvec + nrhs) + (double)L.g.V / L.g.bvol * 2 * L.nvec * s * nrhs,
        frac * (double)L.n() * 8.0 * L.nvec * nrhs,
        launch_restrict<R>(coarse, fine, Prec<R>::vecs(c, L), L.g.V, L.nc, L.g.bvol, L.nvec, nrhs, L.fine, c->st,
                           face, L.g.b));
}
template <typename R>
static void prolong_op(wcmg_ctx* c, int l, cplx<R>* fine, const cplx<R>* coarse, int nrhs) {
  Level& L = c->L[l];
  if (!L.have_P) throw Error(WCMG_ERR_STATE, "prolongator of level not built");
  if (!c->capturing) c->opc[WCMG_OPC_PROLONG][l] += nrhs;
  const double s = sizeof(cplx<R>);
  KPROF(c, WCMG_K_PROLONG, (double)L.n() * s * (L.nvec + nrhs) + (double)L.g.V / L.g.bvol * 2 * L.nvec * s * nrhs,
        (double)L.n() * 8.0 * L.nvec * nrhs,
        launch_prolong<R>(fine, coarse, Prec<R>::vecs(c, L), L.g.V, L.nc, L.g.bvol, L.nvec, nrhs, L.fine, c->st));
}

template <typename R>
static void copy_fields(wcmg_ctx* c, cplx<R>* dst, const cplx<R>* src, long long n) {
  if (c->capturing) launch_copy_idx<R>(dst, src, n, nullptr, 0, 0, c->st);  // kernel node, legal in any body
  else WCMG_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * sizeof(cplx<R>), cudaMemcpyDeviceToDevice, c->st));
}

// ---------------- BLAS wrappers (profiled) ----------------
template <typename R>
static void norm2_op(wcmg_ctx* c, double* out, const cplx<R>* a, long long n, int nrhs) {
  KPROF(c, WCMG_K_BLAS, (double)n * nrhs * sizeof(cplx<R>), 4.0 * n * nrhs,
        launch_norm2<R>(out, a, n, nrhs, c->partial_d.p, c->st));
}
template <typename R>
static void dot_op(wcmg_ctx* c, double2* out, const cplx<R>* a, const cplx<R>* b, long long n, int nrhs) {
  KPROF(c, WCMG_K_BLAS, 2.0 * n * nrhs * sizeof(cplx<R>), 8.0 * n * nrhs,
        launch_dot<R>(out, a, b, n, nrhs, c->partial.p, c->st));
}

// ---------------- MR (smoother) ----------------
// Sec. 2.1 MinimalResidual, zero initial guess, fixed number of steps:
//   r = b; k times: p = A r, alpha = <p, r>/<p, p>, x += alpha r, r -= alpha p.
template <typename R>
static void mr(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs, int steps) {
  Level& L = c->L[l];
  const long long n = L.n();
  cplx<R>* r = ws<R>(L, "mr_r", nrhs);
  cplx<R>* p = ws<R>(L, "mr_p", nrhs);
  L.sc.ensure(max_rhs_all(c), std::max(c->p.outer_restart, c->p.coarse_restart));
  if (steps == 0) {
    launch_fill_zero<R>(x, n * nrhs, c->st);
    return;
  }
  // the first step reads b as its residual and sets x = alpha r; the last one leaves r
  for (int k = 0; k < steps; ++k) {
    const cplx<R>* rk = k == 0 ? b : r;
    if (l == 0) {
      // fine level: the two reductions come out of the Dslash epilogue
      if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
      const long long np = (long long)max_rhs_all(c) * dslash_partials(L.g.V);
      c->mr_pr.ensure(np);
      c->mr_pp.ensure(np);
      const double V = L.g.V, s = sizeof(cplx<R>);
      const int cls = sizeof(R) == 8 ? WCMG_K_DSLASH64 : WCMG_K_DSLASH;
      if (!c->capturing) c->opc[WCMG_OPC_APPLY][0] += nrhs;
      KPROF(c, cls, V * s * (24.0 * nrhs + 72.0), V * (1872.0 + 16.0) * nrhs,
            launch_dslash_mr<R>(p, rk, Prec<R>::gauge(c), Prec<R>::clover(c), L.g.lg(), nrhs, L.sc.pr(),
                                L.sc.slot(4), c->mr_pr.p, c->mr_pp.p, c->st));
    } else {
      apply_op<R>(c, l, p, rk, nrhs);
      dot_op<R>(c, L.sc.pr(), p, rk, n, nrhs);
      norm2_op<R>(c, L.sc.slot(4), p, n, nrhs);
    }
    const bool first = k == 0, last = k + 1 == steps;
    KPROF(c, WCMG_K_BLAS, ((first ? 2.0 : 3.0) + (last ? 0.0 : 2.0)) * n * nrhs * sizeof(cplx<R>),
          16.0 * n * nrhs,
          launch_mr_update<R>(x, r, p, L.sc.pr(), L.sc.slot(4), n, nrhs, c->st, first, !last, rk));
  }
}

template <typename R> static void cycle(wcmg_ctx* c, int l, cplx<R>* e, const cplx<R>* r, int nrhs);
template <typename R> static void smooth(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs);

// ---------------- (F)GMRES ----------------
struct KrylovOut {
  int iterations = 0;
  bool converged = false;
};

// Batched right-preconditioned flexible GMRES(m) on level l (GMRES when
// precond = false).  Arnoldi by classical Gram-Schmidt applied twice (CGS2,
// equal to modified Gram-Schmidt in exact arithmetic), complex Givens
// rotations and the least-squares update in FP64 on the device.  Each rhs stops
// when its recurrence residual is <= tol * ||b||; with verify the true residual
// b - A x decides at the end of a cycle.  max_cycles = 0: unlimited restarts.
template <typename R>
static KrylovOut fgmres(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs, int m, double tol, int maxiter,
                        bool x_zero, bool verify, bool precond, int max_cycles = 0,
                        LevelScalars* scp = nullptr) {
  Level& L = c->L[l];
  LevelScalars& SC = scp ? *scp : L.sc;
  const long long n = L.n();
  const int mr_ = max_rhs_all(c);
  SC.ensure(mr_, std::max(m, std::max(c->p.outer_restart, c->p.coarse_restart)));
  cplx<R>* Vb = ws<R>(L, precond ? "fg_V" : "gm_V", (long long)(m + 1) * nrhs);
  cplx<R>* Zb = precond ? ws<R>(L, "fg_Z", (long long)m * nrhs) : nullptr;
  cplx<R>* w = ws<R>(L, precond ? "fg_w" : "gm_w", nrhs);
  cplx<R>* r = ws<R>(L, precond ? "fg_r" : "gm_r", nrhs);
  const long long bstride = n * nrhs;
  GmresState S = SC.state(m);
  const int ldh = m + 1;
  norm2_op<R>(c, S.bnorm, b, n, nrhs);
  launch_sqrt_inplace(S.bnorm, nrhs, c->st);
  WCMG_CUDA(cudaMemsetAsync(S.done, 0, sizeof(int) * nrhs, c->st));
  if (x_zero) {
    launch_fill_zero<R>(x, n * nrhs, c->st);
    copy_fields<R>(c, r, b, n * nrhs);
  } else {
    apply_op<R>(c, l, r, x, nrhs);
    launch_axpby<R>(r, 1.0, b, -1.0, n, nrhs, c->st);  // r = b - A x
  }
  KrylovOut out;
  int cycles = 0;
  norm2_op<R>(c, SC.slot(1), r, n, nrhs);
  while (true) {
    launch_gmres_start(S, SC.slot(1), tol, nrhs, SC.slot(2), c->st);
    launch_scale_dev<R>(Vb, r, SC.slot(2), 0, n, nrhs, c->st);
    int steps = 0;
    std::vector<double> prev_res;
    if (precond && l == 0 && c->learned_on) {
      const double* rs = read_doubles(c, S.resid, nrhs);
      prev_res.assign(rs, rs + nrhs);
    }
    const int* act = read_ints(c, S.active, nrhs);
    bool any = false;
    for (int q = 0; q < nrhs; ++q) any |= act[q] != 0;
    for (int j = 0; j < m && any; ++j) {
      cplx<R>* vj = Vb + (long long)j * bstride;
      cplx<R>* z = vj;
      if (precond) {
        z = Zb + (long long)j * bstride;
        cycle<R>(c, l, z, vj, nrhs);
      }
      apply_op<R>(c, l, w, z, nrhs);
      if (arnoldi_fused_ok(n, nrhs, m)) {
        KPROF(c, WCMG_K_KRYLOV, (4.0 * (j + 1) + 6.0) * n * sizeof(cplx<R>), 32.0 * (j + 1) * n,
              launch_arnoldi_fused<R>(Vb, bstride, w, n, S, j, nullptr, tol, verify ? 0 : 1, c->st));
      } else {
        KPROF(c, WCMG_K_KRYLOV, (double)(j + 2) * n * nrhs * sizeof(cplx<R>), 8.0 * (j + 1) * n * nrhs,
              launch_multidot<R>(SC.h1(), Vb, bstride, j + 1, ldh, w, n, nrhs, c->partial.p, c->st));
        KPROF(c, WCMG_K_KRYLOV, (double)(j + 3) * n * nrhs * sizeof(cplx<R>), 8.0 * (j + 1) * n * nrhs,
              launch_multiaxpy<R>(w, Vb, bstride, j + 1, SC.h1(), ldh, -1.0, n, nrhs, c->st));
        KPROF(c, WCMG_K_KRYLOV, (double)(j + 2) * n * nrhs * sizeof(cplx<R>), 8.0 * (j + 1) * n * nrhs,
              launch_multidot<R>(SC.h2(), Vb, bstride, j + 1, ldh, w, n, nrhs, c->partial.p, c->st));
        KPROF(c, WCMG_K_KRYLOV, (double)(j + 3) * n * nrhs * sizeof(cplx<R>), 8.0 * (j + 1) * n * nrhs,
              launch_multiaxpy<R>(w, Vb, bstride, j + 1, SC.h2(), ldh, -1.0, n, nrhs, c->st));
        norm2_op<R>(c, SC.slot(0), w, n, nrhs);
        launch_gmres_step(S, j, SC.h1(), SC.h2(), SC.slot(0), tol, verify ? 0 : 1, nrhs, SC.slot(3), c->st);
        launch_scale_dev<R>(Vb + (long long)(j + 1) * bstride, w, SC.slot(3), 0, n, nrhs, c->st);
      }
      ++steps;
      ++out.iterations;
      if (precond && l == 0 && c->learned_on && c->coarse_mode == WCMG_COARSE_LEARNED) {
        // plain multigrid judges the learned correction: fall back when an outer
        // iteration reduces the residual estimate by less than fallback_ratio
        const double* rs = read_doubles(c, S.resid, nrhs);
        double worst = 0.0;
        for (int q = 0; q < nrhs; ++q) {
          const double prev = prev_res.size() == (size_t)nrhs ? prev_res[q] : 0.0;
          if (prev > 0.0) worst = std::max(worst, rs[q] / prev);
        }
        prev_res.assign(rs, rs + nrhs);
        if (c->fallback_ratio > 0.0 && worst > c->fallback_ratio) {
          c->learned_on = false;
          c->learned_fallback = true;
        }
      }
      act = read_ints(c, S.active, nrhs);
      any = false;
      for (int q = 0; q < nrhs; ++q) any |= act[q] != 0;
      if (out.iterations >= maxiter) break;
    }
    ++cycles;
    if (steps > 0) {
      launch_gmres_solve_y(S, nrhs, c->st);
      KPROF(c, WCMG_K_KRYLOV, (double)(steps + 2) * n * nrhs * sizeof(cplx<R>), 8.0 * steps * n * nrhs,
            launch_multiaxpy<R>(x, precond ? Zb : Vb, bstride, steps, S.y, m, 1.0, n, nrhs, c->st));
    }
    if (max_cycles > 0 && cycles >= max_cycles) {
      out.converged = false;
      return out;
    }
    const int* dn = read_ints(c, S.done, nrhs);
    bool all = true;
    for (int q = 0; q < nrhs; ++q) all &= dn[q] != 0;
    if (all && !verify) { out.converged = true; return out; }
    apply_op<R>(c, l, r, x, nrhs);
    launch_axpby<R>(r, 1.0, b, -1.0, n, nrhs, c->st);
    norm2_op<R>(c, SC.slot(1), r, n, nrhs);
    launch_gmres_mark_done(S, SC.slot(1), tol, nrhs, c->st);
    const double* nr = read_doubles(c, SC.slot(1), nrhs);
    for (int q = 0; q < nrhs; ++q)
      if (!std::isfinite(nr[q])) throw Error(WCMG_ERR_NAN, "non-finite residual in Krylov solver");
    dn = read_ints(c, S.done, nrhs);
    all = true;
    for (int q = 0; q < nrhs; ++q) all &= dn[q] != 0;
    if (all) { out.converged = true; return out; }
    if (out.iterations >= maxiter || steps == 0) return out;
  }
}

// ---------------- device-driven (F)GMRES for CUDA-graph capture ----------------
// The same algorithm as fgmres() above, with every stopping test taken on the
// device by the control kernels of graph.cu: the Arnoldi loop and the restart
// loop become conditional WHILE nodes, the true-residual step of a restart an IF
// node.  Kernels that depend on the step number j read it from KCtl::j.  Only
// used while the context is capturing a graph.

static cudaGraphConditionalHandle cond_handle(wcmg_ctx* c) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  WCMG_CUDA(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) throw Error(WCMG_ERR_STATE, "graph handle outside a capture");
  cudaGraphConditionalHandle h;
  WCMG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  return h;
}

static BodyCount body_count(wcmg_ctx* c, int slot) { return BodyCount{c->body_counts.p, slot, c->gstat.p}; }

// Append a conditional node (WHILE or IF, condition h) to the capturing stream and
// capture body(slot) into its body graph on the next capture stream.
template <class F>
static void cond_node(wcmg_ctx* c, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, F&& body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  WCMG_CUDA(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, &deps, &edges, &nd));
  if (cs != cudaStreamCaptureStatusActive) throw Error(WCMG_ERR_STATE, "conditional node outside a capture");
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  WCMG_CUDA(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
  WCMG_CUDA(cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t bodyg = np.conditional.phGraph_out[0];
  if (c->cap_depth + 1 >= wcmg_ctx::MAX_CAP_DEPTH) throw Error(WCMG_ERR_STATE, "graph nesting too deep");
  if ((int)c->body_counts_h.size() >= wcmg_ctx::MAX_BODIES) throw Error(WCMG_ERR_STATE, "too many graph bodies");
  const int slot = (int)c->body_counts_h.size();
  c->body_counts_h.push_back(0);
  cudaStream_t& bs = c->cap_st[c->cap_depth + 1];
  if (!bs) WCMG_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
  cudaStream_t parent = c->st;
  WCMG_CUDA(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  ++c->cap_depth;
  c->st = bs;
  const long long l0 = launch_counter();
  c->nested.push_back(0);
  try {
    body(slot);
  } catch (...) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(bs, &dummy);
    c->st = parent;
    --c->cap_depth;
    c->nested.pop_back();
    throw;
  }
  const long long total = launch_counter() - l0;
  const long long inner = c->nested.back();
  c->nested.pop_back();
  c->body_counts_h[slot] = (int)(total - inner);
  if (!c->nested.empty()) c->nested.back() += total;
  cudaGraph_t dummy = nullptr;
  WCMG_CUDA(cudaStreamEndCapture(bs, &dummy));
  c->st = parent;
  --c->cap_depth;
}

template <typename R>
static void fgmres_g(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs, int m, double tol, int maxiter,
                     bool x_zero, bool verify, bool precond, int max_cycles, KCtl* K, const int* budget_its,
                     int budget_max, long long* acc, LevelScalars* scp = nullptr) {
  Level& L = c->L[l];
  LevelScalars& SC = scp ? *scp : L.sc;
  const long long n = L.n();
  SC.ensure(max_rhs_all(c), std::max(m, std::max(c->p.outer_restart, c->p.coarse_restart)));
  cplx<R>* Vb = ws<R>(L, precond ? "fg_V" : "gm_V", (long long)(m + 1) * nrhs);
  cplx<R>* Zb = precond ? ws<R>(L, "fg_Z", (long long)m * nrhs) : nullptr;
  cplx<R>* w = ws<R>(L, precond ? "fg_w" : "gm_w", nrhs);
  cplx<R>* r = ws<R>(L, precond ? "fg_r" : "gm_r", nrhs);
  cplx<R>* vcur = ws<R>(L, precond ? "fg_vc" : "gm_vc", nrhs);
  cplx<R>* zcur = precond ? ws<R>(L, "fg_zc", nrhs) : nullptr;
  const long long bstride = n * nrhs;
  GmresState S = SC.state(m);
  const int ldh = m + 1;
  const int* jd = &K->j;
  norm2_op<R>(c, S.bnorm, b, n, nrhs);
  launch_sqrt_inplace(S.bnorm, nrhs, c->st);
  launch_fill_int(S.done, 0, nrhs, c->st);
  if (x_zero) {
    launch_fill_zero<R>(x, n * nrhs, c->st);
    copy_fields<R>(c, r, b, n * nrhs);
  } else {
    apply_op<R>(c, l, r, x, nrhs);
    launch_axpby<R>(r, 1.0, b, -1.0, n, nrhs, c->st);  // r = b - A x
  }
  norm2_op<R>(c, SC.slot(1), r, n, nrhs);
  const bool single = max_cycles == 1;
  const cudaGraphConditionalHandle h_loop = single ? 0 : cond_handle(c);
  launch_kctl_init(K, maxiter, budget_its, budget_max, h_loop, single ? 0 : 1, c->st);

  // one restart cycle: Arnoldi steps while any rhs is active, then x += Z y
  auto one_cycle = [&]() {
    launch_gmres_start(S, SC.slot(1), tol, nrhs, SC.slot(2), c->st);
    launch_scale_dev<R>(Vb, r, SC.slot(2), 0, n, nrhs, c->st);
    const cudaGraphConditionalHandle h_arn = cond_handle(c);
    launch_kctl_cycle_begin(K, S.active, nrhs, m, h_arn, c->st);
    cond_node(c, h_arn, cudaGraphCondTypeWhile, [&](int slot) {
      launch_copy_idx<R>(vcur, Vb, bstride, jd, 0, bstride, c->st);  // vcur = V_j
      const cplx<R>* z = vcur;
      if (precond) {
        cycle<R>(c, l, zcur, vcur, nrhs);
        launch_copy_idx<R>(Zb, zcur, bstride, jd, bstride, 0, c->st);  // Z_j = M V_j
        z = zcur;
      }
      apply_op<R>(c, l, w, z, nrhs);
      if (arnoldi_fused_ok(n, nrhs, m)) {
        KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
              launch_arnoldi_fused<R>(Vb, bstride, w, n, S, 0, jd, tol, verify ? 0 : 1, c->st));
      } else {
        KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
              launch_multidot<R>(SC.h1(), Vb, bstride, m, ldh, w, n, nrhs, c->partial.p, c->st, jd, 1));
        KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
              launch_multiaxpy<R>(w, Vb, bstride, m, SC.h1(), ldh, -1.0, n, nrhs, c->st, jd, 1));
        KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
              launch_multidot<R>(SC.h2(), Vb, bstride, m, ldh, w, n, nrhs, c->partial.p, c->st, jd, 1));
        KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
              launch_multiaxpy<R>(w, Vb, bstride, m, SC.h2(), ldh, -1.0, n, nrhs, c->st, jd, 1));
        norm2_op<R>(c, SC.slot(0), w, n, nrhs);
        launch_gmres_step(S, 0, SC.h1(), SC.h2(), SC.slot(0), tol, verify ? 0 : 1, nrhs, SC.slot(3), c->st,
                          jd);
        launch_scale_dev<R>(Vb, w, SC.slot(3), 0, n, nrhs, c->st, jd, 1, bstride);  // V_{j+1}
      }
      launch_kctl_step_end(K, S.active, nrhs, m, acc, body_count(c, slot), h_arn, c->st);
    });
    launch_gmres_solve_y(S, nrhs, c->st);
    KPROF(c, WCMG_K_KRYLOV, 0.0, 0.0,
          launch_multiaxpy<R>(x, precond ? Zb : Vb, bstride, m, S.y, m, 1.0, n, nrhs, c->st, jd, 0));
  };

  if (single) {  // one cycle, no restart loop (the FP32 cycles of the mixed solve)
    one_cycle();
    return;
  }
  cond_node(c, h_loop, cudaGraphCondTypeWhile, [&](int slot_r) {
    one_cycle();
    const cudaGraphConditionalHandle h_if = cond_handle(c);
    launch_kctl_cycle_end(K, S.done, nrhs, verify ? 1 : 0, max_cycles, body_count(c, slot_r), h_if, c->st);
    int slot_if = -1;
    cond_node(c, h_if, cudaGraphCondTypeIf, [&](int slot_i) {
      slot_if = slot_i;
      apply_op<R>(c, l, r, x, nrhs);
      launch_axpby<R>(r, 1.0, b, -1.0, n, nrhs, c->st);
      norm2_op<R>(c, SC.slot(1), r, n, nrhs);
      launch_gmres_mark_done(S, SC.slot(1), tol, nrhs, c->st);
    });
    launch_kctl_restart_check(K, S.done, SC.slot(1), nrhs, body_count(c, slot_if), h_loop, c->st);
  });
}

// ---------------- smoother ----------------
// S_k(D_l; b) from a zero initial guess: MR(k), or GMRES with k steps (no restart,
// no tolerance) on the level's own Krylov state, so that it can run inside the
// outer FGMRES on the same level.
template <typename R>
static void sap(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs, int steps, int cycles);

template <typename R>
static void smooth(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs) {
  const int k = c->p.smoother_steps;
  if (c->p.smoother == WCMG_SMOOTHER_MR || k == 0) {
    mr<R>(c, l, x, b, nrhs, k);
    return;
  }
  if (c->p.smoother == WCMG_SMOOTHER_SAP) {
    sap<R>(c, l, x, b, nrhs, k, c->p.sap_cycles);
    return;
  }
  Level& L = c->L[l];
  if (c->capturing)
    fgmres_g<R>(c, l, x, b, nrhs, k, 0.0, k, true, false, false, 1, c->kctl.p + 2 + WCMG_MAX_LEVELS + l, nullptr, 0,
                nullptr, &L.sc_s);
  else
    fgmres<R>(c, l, x, b, nrhs, k, 0.0, k, true, false, false, 1, &L.sc_s);
}

// SAP (Sec. 4): from x = 0, `cycles` times, for colour c = 0 then 1:
//   r = b - D x on the blocks of colour c (0 elsewhere);
//   `steps` block-local MR steps on D_B (D without the hops leaving a block), one
//   step length per block, the steps added to x.
// D x is needed on the blocks of colour c only (the fine stencil skips the others).
// Fine level with aggregates of <= 256 sites: the steps of a pass run fused, one CTA
// per block (launch_sap_fine).  Otherwise each step is one block-interior stencil and
// one fused block-reduction + update kernel (D_B r vanishes where r does).
template <typename R>
static void sap(wcmg_ctx* c, int l, cplx<R>* x, const cplx<R>* b, int nrhs, int steps, int cycles) {
  Level& L = c->L[l];
  if (!L.colour.p) throw Error(WCMG_ERR_STATE, "SAP needs the level's aggregates");
  if (l == 0 && !c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  const long long n = L.n();
  const bool fused = l == 0 && sap_fine_threads(L.g.bvol) != 0;
  cplx<R>* r = fused ? nullptr : ws<R>(L, "sap_r", nrhs);
  cplx<R>* p = ws<R>(L, "sap_p", nrhs);
  const double s = sizeof(cplx<R>);
  const int cls = sizeof(R) == 8 ? WCMG_K_DSLASH64 : WCMG_K_DSLASH;
  launch_fill_zero<R>(x, n * nrhs, c->st);
  for (int cyc = 0; cyc < cycles; ++cyc)
    for (int col = 0; col < 2; ++col) {
      const bool x_zero = cyc == 0 && col == 0;
      const double sites = (double)L.sap_count[col] * L.g.bvol;
      if (!x_zero) {
        if (l == 0)
          KPROF(c, cls, sites * s * (24.0 * nrhs + 72.0), sites * 1872.0 * nrhs,
                launch_dslash<R>(p, x, Prec<R>::gauge(c), Prec<R>::clover(c), L.g.lg(), nrhs, ST_FULL, 0, c->st,
                                 L.colour.p, col));
        else
          apply_op<R>(c, l, p, x, nrhs);
      }
      if (fused && c->p.sap_eo) {
        KPROF(c, cls, sites * s * ((x_zero ? 36.0 : 48.0) * nrhs + 108.0), sites * (steps + 1) * 1900.0 * nrhs,
              launch_sap_fine_eo<R>(x, b, x_zero ? nullptr : p, Prec<R>::gauge(c), Prec<R>::clover(c),
                                    Prec<R>::clover_inv(c), L.g.lg(), L.sap_list.p + (col ? L.sap_count[0] : 0),
                                    L.opar.p, L.sap_count[col], steps, nrhs, c->st));
        continue;
      }
      if (fused) {
        KPROF(c, cls, sites * s * ((x_zero ? 36.0 : 48.0) * nrhs + 72.0), sites * steps * 1900.0 * nrhs,
              launch_sap_fine<R>(x, b, x_zero ? nullptr : p, Prec<R>::gauge(c), Prec<R>::clover(c), L.g.lg(),
                                 L.sap_list.p + (col ? L.sap_count[0] : 0), L.sap_count[col], steps, nrhs, c->st));
        continue;
      }
      KPROF(c, WCMG_K_BLAS, (x_zero ? 1.5 : 2.0) * n * nrhs * s, 1.0 * n * nrhs,
            launch_sap_residual<R>(r, b, x_zero ? nullptr : p, L.colour.p, col, L.g.V, L.nc, L.g.bvol, L.fine, nrhs,
                                   c->st));
      for (int k = 0; k < steps; ++k) {
        apply_op<R>(c, l, p, r, nrhs, ST_BLOCK_INTERIOR);
        KPROF(c, WCMG_K_BLAS, 2.5 * n * nrhs * s, 12.0 * n * nrhs,
              launch_sap_block_mr<R>(x, r, p, L.colour.p, col, L.g.V, L.nc, L.g.bvol, L.fine, nrhs, c->st));
      }
    }
}

// ---------------- learned coarse correction (PTC network) ----------------
constexpr int PTC_NW1 = WCMG_PTC_HIDDEN * 1 * 9 * 16;
constexpr int PTC_NW2 = 1 * WCMG_PTC_HIDDEN * 9 * 16;

static void ptc_layer_fwd(wcmg_ctx* c, float2* out, const float2* in, const float2* W, int nin, int nout, int nrhs) {
  Level& L = c->L[0];
  const double V = L.g.V;
  KPROF(c, WCMG_K_PTC, V * 96.0 * (nin + nout) * nrhs + 8.0 * V * 72.0 * 4,
        V * 8.0 * (double)nin * nout * 9 * (48 + 36) * nrhs,
        launch_ptc_forward(out, in, W, c->gauge32.p, L.g.d_nbr.p, L.g.V, nin, nout, nrhs, c->st));
}

// out = N(in), FP32, nrhs fields in the internal fine layout
static void ptc_forward(wcmg_ctx* c, float2* out, const float2* in, int nrhs) {
  if (!c->have_ptc) throw Error(WCMG_ERR_STATE, "PTC weights not set");
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  float2* hid = ws<float>(c->L[0], "ptc_hid", (long long)WCMG_PTC_HIDDEN * nrhs);
  ptc_layer_fwd(c, hid, in, c->ptcW.p, 1, WCMG_PTC_HIDDEN, nrhs);
  ptc_layer_fwd(c, out, hid, c->ptcW.p + PTC_NW1, WCMG_PTC_HIDDEN, 1, nrhs);
}

// Gradients dL/d conj(W) into ptcG (summed over the fields) and, if gin is not
// null, dL/d conj(in), given gout = dL/d conj(N(in)).
static void ptc_backward(wcmg_ctx* c, const float2* in, const float2* gout, float2* gin, int nrhs) {
  Level& L = c->L[0];
  const int V = L.g.V, H = WCMG_PTC_HIDDEN;
  float2* hid = ws<float>(L, "ptc_hid", (long long)H * nrhs);
  float2* ghid = ws<float>(L, "ptc_ghid", (long long)H * nrhs);
  ptc_layer_fwd(c, hid, in, c->ptcW.p, 1, H, nrhs);
  c->ptcPartial.ensure((size_t)std::max(ptc_wgrad_partial_size(V, H, 1, nrhs), ptc_wgrad_partial_size(V, 1, H, nrhs)));
  const double flops = (double)V * 8.0 * H * 9 * (48 + 36) * nrhs;
  KPROF(c, WCMG_K_PTC, (double)V * 96.0 * (H + 1) * nrhs, flops,
        launch_ptc_wgrad(c->ptcG.p + PTC_NW1, c->ptcPartial.p, gout, hid, c->gauge32.p, L.g.d_nbr.p, V, H, 1, nrhs,
                         c->st));
  KPROF(c, WCMG_K_PTC, (double)V * 96.0 * (H + 1) * nrhs, flops,
        launch_ptc_backward_data(ghid, gout, c->ptcW.p + PTC_NW1, c->gauge32.p, L.g.d_nbr.p, V, H, 1, nrhs, c->st));
  KPROF(c, WCMG_K_PTC, (double)V * 96.0 * (H + 1) * nrhs, flops,
        launch_ptc_wgrad(c->ptcG.p, c->ptcPartial.p, ghid, in, c->gauge32.p, L.g.d_nbr.p, V, 1, H, nrhs, c->st));
  if (gin)
    KPROF(c, WCMG_K_PTC, (double)V * 96.0 * (H + 1) * nrhs, flops,
          launch_ptc_backward_data(gin, ghid, c->ptcW.p, c->gauge32.p, L.g.d_nbr.p, V, 1, H, nrhs, c->st));
}

static void ptc_alloc(wcmg_ctx* c) {
  c->ptcW.ensure(WCMG_PTC_NWEIGHTS);
  c->ptcG.ensure(WCMG_PTC_NWEIGHTS);
  c->ptcM.ensure(WCMG_PTC_NWEIGHTS);
  c->ptcV.ensure(WCMG_PTC_NWEIGHTS);
}

// ---------------- multigrid cycle ----------------
// M_l(r): e = P_l CoarseSolve_{l+1}(P_l^dag r); e += MR_k(D_l; r - D_l e).
// CoarseSolve is GMRES at the coarsest level and one cycle of level l+1 between.
// The coarsest solve: GMRES on D_c, or with params.coarse_eo on the odd-site Schur
// complement: b^_o = [b - D A_ee^-1 b_e]_o, GMRES on S to the coarse tolerance of
// ||b^_o||, x_e = A_ee^-1 [b - D x_o]_e.
template <typename R>
static void coarsest_gmres(wcmg_ctx* c, int lc, cplx<R>* x, const cplx<R>* b, int nrhs, bool x0) {
  if (c->capturing) {
    fgmres_g<R>(c, lc, x, b, nrhs, c->p.coarse_restart, c->p.coarse_tol, c->p.coarse_maxiter, !x0, false, false, 0,
                c->kctl.p + 2 + lc, nullptr, 0, c->gstat.p + 1);
  } else {
    KrylovOut k = fgmres<R>(c, lc, x, b, nrhs, c->p.coarse_restart, c->p.coarse_tol, c->p.coarse_maxiter, !x0, false,
                            false);
    c->coarse_its += k.iterations;
  }
}
template <typename R>
static void coarsest_solve(wcmg_ctx* c, int lc, cplx<R>* x, const cplx<R>* b, int nrhs, bool x0) {
  if (!c->p.coarse_eo) {
    coarsest_gmres<R>(c, lc, x, b, nrhs, x0);
    return;
  }
  Level& C = c->L[lc];
  ensure_ainv(c, lc);
  const int nb = C.nc;
  const unsigned char* par = C.g.d_par.p;
  cplx<R>* bh = ws<R>(C, "eo_b", nrhs);
  cplx<R>* u = ws<R>(C, "eo_u", nrhs);
  cplx<R>* y = ws<R>(C, "eo_y", nrhs);
  KPROF(c, WCMG_K_COARSE, 0.0, 0.0,
        launch_blockinv_apply<R>(u, b, ainv_of<R>(C), par, 0, C.g.V, nb, nrhs, c->st));  // A_ee^-1 b_e
  apply_parity<R>(c, lc, y, u, nrhs, 1);                                             // [D A_ee^-1 b_e]_o
  launch_parity_axpy<R>(bh, b, y, -1.0, par, 1, C.g.V, nb, nrhs, c->st);             // b^_o
  if (x0) launch_parity_axpy<R>(x, x, x, 0.0, par, 1, C.g.V, nb, nrhs, c->st);        // odd part of the guess
  c->eo_schur = true;
  try {
    coarsest_gmres<R>(c, lc, x, bh, nrhs, x0);
  } catch (...) {
    c->eo_schur = false;
    throw;
  }
  c->eo_schur = false;
  apply_parity<R>(c, lc, y, x, nrhs, 0);                                             // [D x_o]_e
  launch_parity_axpy<R>(u, b, y, -1.0, par, 0, C.g.V, nb, nrhs, c->st);              // [b - D x_o]_e
  KPROF(c, WCMG_K_COARSE, 0.0, 0.0,
        launch_blockinv_apply<R>(y, u, ainv_of<R>(C), par, 0, C.g.V, nb, nrhs, c->st));  // x_e
  launch_axpby<R>(x, 1.0, y, 1.0, C.n(), nrhs, c->st);
}

template <typename R>
static void cycle(wcmg_ctx* c, int l, cplx<R>* e, const cplx<R>* r, int nrhs) {
  Level& L = c->L[l];
  Level& C = c->L[l + 1];
  const long long n = L.n();
  const bool learned = sizeof(R) == 4 && l == 0 && c->learned_on;
  if (learned && c->coarse_mode == WCMG_COARSE_LEARNED) {
    // learned coarse correction in place of P CoarseSolve(P^dag r)
    ptc_forward(c, (float2*)e, (const float2*)r, nrhs);
    ++c->learned_cycles;
  } else {
    cplx<R>* rc = ws<R>(C, "cyc_rc", nrhs);
    cplx<R>* ec = ws<R>(C, "cyc_ec", nrhs);
    restrict_op<R>(c, l, rc, r, nrhs);
    if (l + 1 == c->p.n_levels - 1) {
      bool x0 = false;
      if (learned && c->coarse_mode == WCMG_COARSE_WARMSTART) {
        // initial guess of the coarsest GMRES: P^dag N(r)
        cplx<R>* t = ws<R>(L, "cyc_ptc", nrhs);
        ptc_forward(c, (float2*)t, (const float2*)r, nrhs);
        restrict_op<R>(c, l, ec, t, nrhs);
        ++c->learned_cycles;
        x0 = true;
      }
      coarsest_solve<R>(c, l + 1, ec, rc, nrhs, x0);
    } else if (c->p.kcycle) {
      // K-cycle: a short FGMRES on the intermediate level, preconditioned by its cycle
      const int ks = c->p.kcycle_steps;
      if (c->capturing)
        fgmres_g<R>(c, l + 1, ec, rc, nrhs, ks, c->p.kcycle_tol, ks, true, false, true, 1, c->kctl.p + 2 + (l + 1),
                    nullptr, 0, nullptr);
      else
        fgmres<R>(c, l + 1, ec, rc, nrhs, ks, c->p.kcycle_tol, ks, true, false, true, 1);
    } else {
      cycle<R>(c, l + 1, ec, rc, nrhs);
    }
    prolong_op<R>(c, l, e, ec, nrhs);
  }
  cplx<R>* t = ws<R>(L, "cyc_t", nrhs);
  cplx<R>* s = ws<R>(L, "cyc_s", nrhs);
  apply_op<R>(c, l, t, e, nrhs);
  launch_axpby<R>(t, 1.0, r, -1.0, n, nrhs, c->st);  // t = r - D e
  smooth<R>(c, l, s, t, nrhs);
  launch_axpby<R>(e, 1.0, s, 1.0, n, nrhs, c->st);
}

// ---------------- setup ----------------
template <typename R>
static void coarsen_body(wcmg_ctx* c, int l) {
  Level& F = c->L[l];
  Level& C = c->L[l + 1];
  const int nb = 2 * F.nvec, Vc = C.g.V;
  const long long nl = (long long)Vc * nb * links_ld(nb);
  cplx<R>* links;
  if (sizeof(R) == 8) {
    links = (cplx<R>*)C.L64.ensure(nl);
    C.op64 = true;
    C.L32_valid = false;
  } else {
    links = (cplx<R>*)C.L32.ensure(nl);
    C.op64 = false;
    C.L32_valid = true;
  }
  WCMG_CUDA(cudaMemsetAsync(links, 0, (size_t)nl * sizeof(cplx<R>), c->st));
  const int chunk = std::min(nb, 48);
  cplx<R>* T = ws<R>(F, "co_T", chunk);
  cplx<R>* res = ws<R>(C, "co_res", chunk);
  if (F.fine) {
    // fine level: both chirality columns of each vector from one stencil pass
    if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
    const int vchunk = chunk / 2;
    const cplx<R>* vecs = Prec<R>::vecs(c, F);
    const double V = F.g.V, s = sizeof(cplx<R>);
    for (int i0 = 0; i0 < F.nvec; i0 += vchunk) {
      const int nv = std::min(vchunk, F.nvec - i0);
      for (int dm = 0; dm < 9; ++dm) {
        const int mode = dm == 0 ? ST_BLOCK_INTERIOR : ST_FACE_HOP;
        const int hop = dm == 0 ? 0 : dm - 1;
        const double frac = dm == 0 ? 1.0 : 1.0 / F.g.b[hop >> 1];
        KPROF(c, sizeof(R) == 8 ? WCMG_K_DSLASH64 : WCMG_K_DSLASH, frac * V * s * (36.0 * nv + 72.0),
              frac * V * 1872.0 * 2 * nv,
              launch_dslash_chiral<R>(T, vecs + (long long)i0 * F.n(), Prec<R>::gauge(c), Prec<R>::clover(c),
                                      F.g.lg(), nv, mode, hop, c->st));
        restrict_op<R>(c, l, res, T, 2 * nv, dm == 0 ? -1 : hop);
        const long long half = (long long)nv * Vc * nb;
        KPROF(c, WCMG_K_COARSEN, (double)Vc * nb * nv * 4.0 * sizeof(cplx<R>), 0.0,
              (launch_scatter_links<R, cplx<R>>(links, res, Vc, nb, dm == 0 ? 0 : dm, i0, nv, c->st)));
        KPROF(c, WCMG_K_COARSEN, 0.0, 0.0,
              (launch_scatter_links<R, cplx<R>>(links, res + half, Vc, nb, dm == 0 ? 0 : dm, F.nvec + i0, nv,
                                                c->st)));
      }
    }
  }
  cplx<R>* cols = F.fine ? nullptr : ws<R>(F, "co_cols", chunk);
  for (int b0 = 0; !F.fine && b0 < nb; b0 += chunk) {
    const int ncols = std::min(chunk, nb - b0);
    KPROF(c, WCMG_K_COARSEN, 2.0 * F.n() * ncols * sizeof(cplx<R>), 0.0,
          launch_make_columns<R>(cols, Prec<R>::vecs(c, F), F.g.V, F.nc, F.nvec, b0, ncols, F.fine, c->st));
    for (int dm = 0; dm < 9; ++dm) {
      const int mode = dm == 0 ? ST_BLOCK_INTERIOR : ST_FACE_HOP;
      const int hop = dm == 0 ? 0 : dm - 1;
      apply_op<R>(c, l, T, cols, ncols, mode, hop);
      restrict_op<R>(c, l, res, T, ncols, dm == 0 ? -1 : hop);
      KPROF(c, WCMG_K_COARSEN, (double)Vc * nb * ncols * 2.0 * sizeof(cplx<R>), 0.0,
            (launch_scatter_links<R, cplx<R>>(links, res, Vc, nb, dm == 0 ? 0 : dm, b0, ncols, c->st)));
    }
  }
  C.have_op = true;
  C.ainv_valid = false;
  C.low_valid = false;
  if (sizeof(R) == 4 && (c->p.coarse_link_prec == WCMG_BF16 || c->p.coarse_link_prec == WCMG_F16)) {
    if (c->p.coarse_link_prec == WCMG_BF16) {
      C.Lbf.ensure(nl);
      launch_convert_links<float2, bf16c>(C.Lbf.p, C.L32.p, nl, c->st);
      build_mma_links(c, l + 1);
    } else {
      C.Lh.ensure(nl);
      launch_convert_links<float2, f16c>(C.Lh.p, C.L32.p, nl, c->st);
    }
    C.low_valid = true;
  }
  C.sigma3 = true;  // a Galerkin product: the five-block copies are exact
  build_links5(c, l + 1);
  // the even-odd coarsest solve's self-block inverses follow every new coarsest operator
  // (built here, outside any capture, so that a replayed solve never sees stale ones)
  if (c->p.coarse_eo && l + 1 == c->p.n_levels - 1) ensure_ainv(c, l + 1);
}

template <typename R>
static void coarsen(wcmg_ctx* c, int l) {
  struct Guard {
    wcmg_ctx* c;
    ~Guard() { c->in_coarsen = false; }
  } guard{c};
  c->in_coarsen = true;
  c->opc[WCMG_OPC_COARSEN][l] += 1;
  coarsen_body<R>(c, l);
}

// Block orthonormalisation of L.v64 in place (Sec. 2.2: Q factor per aggregate and
// chirality), in FP64 or, with params.ortho_df, in double-float arithmetic.
static void ortho_level(wcmg_ctx* c, int l, const float2* in32 = nullptr, float2* out32 = nullptr) {
  Level& L = c->L[l];
  const long long n = (long long)L.nvec * L.n();
  WCMG_CUDA(cudaMemsetAsync(c->errflag.p, 0, sizeof(int), c->st));
  c->opc[WCMG_OPC_ORTHO][l] += 1;
  // algorithmic work: one Gram-Schmidt pass, nvec (nvec - 1) complex MAC per panel row
  // (dots + updates); a second pass, when the cancellation test asks for it, is extra.
  if (c->p.ortho_df) {
    float4* qdf = reinterpret_cast<float4*>(ws<double>(L, "ortho_qdf", L.nvec));
    KPROF(c, WCMG_K_ORTHO, 2.0 * n * 16.0, 8.0 * n * (L.nvec - 1),
          launch_block_ortho_df(L.v64.p, qdf, L.g.V, L.nc, L.g.bvol, L.nvec, L.fine, c->errflag.p, c->st, in32,
                                out32));
  } else {
    KPROF(c, WCMG_K_ORTHO, 2.0 * n * 16.0, 8.0 * n * (L.nvec - 1),
          launch_block_ortho(L.v64.p, L.g.V, L.nc, L.g.bvol, L.nvec, L.fine, c->errflag.p, c->st));
  }
  const int* e = read_ints(c, c->errflag.p, 1);
  if (e[0]) throw Error(WCMG_ERR_NAN, "rank-deficient aggregate in block orthonormalisation");
}

// P_l from the level's raw vectors at precision R.
template <typename R>
static void build_P(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  const long long n = (long long)L.nvec * L.n();
  L.v64.ensure(n);
  if constexpr (sizeof(R) == 4) {
    if (c->p.ortho_df) {
      // the double-float kernel reads the FP32 vectors and writes the FP32 copy of P as
      // well: no conversion passes (the same bits as converting before and after)
      L.v32.ensure(n);
      ortho_level(c, l, Prec<R>::raw(L).p, L.v32.p);
      L.v32_valid = true;
      L.have_P = true;
      return;
    }
  }
  launch_convert<R, double>(L.v64.p, Prec<R>::raw(L).p, n, c->st);
  ortho_level(c, l);
  L.v32_valid = false;
  L.have_P = true;
}

// One setup sweep: the smoother applied to the level's raw near-null vectors, whose
// output becomes the new raw vectors.  They are not normalised: the next sweep's
// smoother, the MG cycle of a refinement sweep (coarse solves to a relative tolerance)
// and the block orthonormalisation all map a positively scaled vector to the same
// result scaled alike or (P) unchanged, so a norm and a scaling pass over the Nvec
// fields per sweep would change nothing but rounding.  The buffers are swapped.
template <typename R>
static void smooth_sweep(wcmg_ctx* c, int l) {
  Level& L = c->L[l];
  const int nv = L.nvec;
  auto& raw = Prec<R>::raw(L);
  auto& next = Prec<R>::raw_next(L);
  next.ensure((size_t)nv * L.n());
  smooth<R>(c, l, next.p, raw.p, nv);
  std::swap(raw, next);
}

template <typename R>
static void setup_all(wcmg_ctx* c, const double2* init, wcmg_stats* st) {
  const int nl = c->p.n_levels;
  auto t0 = std::chrono::steady_clock::now();
  long long off = 0;
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = c->L[l];
    auto& raw = Prec<R>::raw(L);
    raw.ensure((size_t)L.nvec * L.n());
    if (L.fine) launch_pack_fine<R>(raw.p, init + off, L.g.d_perm.p, L.g.V, L.nvec, c->st);
    else launch_pack_coarse<R>(raw.p, init + off, L.g.d_perm.p, L.g.V, L.nc, L.nvec, c->st);
    off += (long long)L.nvec * L.n();
    for (int s = 0; s < c->p.setup_init_sweeps; ++s) smooth_sweep<R>(c, l);
    build_P<R>(c, l);
    coarsen<R>(c, l);
  }
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  auto t1 = std::chrono::steady_clock::now();
  for (int s = 0; s < c->p.setup_refine_sweeps; ++s) {
    Level& L = c->L[0];
    const int nv = L.nvec;
    auto& raw = Prec<R>::raw(L);
    auto& next = Prec<R>::raw_next(L);
    next.ensure((size_t)nv * L.n());
    cycle<R>(c, 0, next.p, raw.p, nv);  // not normalised either (see smooth_sweep)
    std::swap(raw, next);
    build_P<R>(c, 0);
    coarsen<R>(c, 0);
    for (int l = 1; l + 1 < nl; ++l) {
      smooth_sweep<R>(c, l);
      build_P<R>(c, l);
      coarsen<R>(c, l);
    }
  }
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  auto t2 = std::chrono::steady_clock::now();
  if (st) {
    st->ms_setup_init = std::chrono::duration<double, std::milli>(t1 - t0).count();
    st->ms_setup_refine = std::chrono::duration<double, std::milli>(t2 - t1).count();
  }
}

// ---------------- outer solve ----------------
static void solve_f64(wcmg_ctx* c, double2* x, const double2* b, int nrhs, wcmg_stats* st) {
  KrylovOut k = fgmres<double>(c, 0, x, b, nrhs, c->p.outer_restart, c->p.outer_tol, c->p.outer_maxiter, !c->guess,
                               true, true);
  st->outer_iterations = k.iterations;
  st->converged = k.converged;
}

// relative tolerance of each FP32 FGMRES cycle between two FP64 defect corrections
constexpr double kInnerTol = 1e-5;

// r = b - D x for the caller's initial guess (c->guess), else x = 0 and r = b (FP64).
static void start_residual(wcmg_ctx* c, double2* x, double2* r, double2* t, const double2* b, int nrhs) {
  const long long n = c->L[0].n();
  if (c->guess) {
    apply_op<double>(c, 0, t, x, nrhs);
    copy_fields<double>(c, r, b, n * nrhs);
    launch_axpby<double>(r, -1.0, t, 1.0, n, nrhs, c->st);
  } else {
    launch_fill_zero<double>(x, n * nrhs, c->st);
    copy_fields<double>(c, r, b, n * nrhs);
  }
}

// Precision change (Sec. 2.1): FP64 iterate and true residual, FP32 FGMRES cycles
// preconditioned by the FP32 multigrid; every restart is a defect correction.
static void solve_mixed(wcmg_ctx* c, double2* x, const double2* b, int nrhs, wcmg_stats* st) {
  Level& L = c->L[0];
  const long long n = L.n();
  double2* r64 = ws<double>(L, "mx_r", nrhs);
  double2* t64 = ws<double>(L, "mx_t", nrhs);
  float2* r32 = ws<float>(L, "mx_r32", nrhs);
  float2* e32 = ws<float>(L, "mx_e32", nrhs);
  L.sc.ensure(max_rhs_all(c), std::max(c->p.outer_restart, c->p.coarse_restart));
  double* bn2 = L.sc.slot(7);
  norm2_op<double>(c, bn2, b, n, nrhs);
  std::vector<double> bnorm(nrhs);
  {
    const double* h = read_doubles(c, bn2, nrhs);
    for (int q = 0; q < nrhs; ++q) bnorm[q] = std::sqrt(h[q]);
  }
  start_residual(c, x, r64, t64, b, nrhs);
  DevBuf<int>& mask = c->errflag;  // errflag has room for max rhs + 1
  std::vector<int> done(nrhs, 0);
  int its = 0, restarts = 0;
  const double inner_tol = kInnerTol;
  while (true) {
    norm2_op<double>(c, L.sc.slot(1), r64, n, nrhs);
    const double* h = read_doubles(c, L.sc.slot(1), nrhs);
    bool all = true;
    double worst = 0;
    for (int q = 0; q < nrhs; ++q) {
      if (!std::isfinite(h[q])) throw Error(WCMG_ERR_NAN, "non-finite residual");
      const double rel = bnorm[q] > 0 ? std::sqrt(h[q]) / bnorm[q] : 0.0;
      worst = std::max(worst, rel);
      done[q] = rel <= c->p.outer_tol;
      all &= done[q] != 0;
    }
    st->true_residual = worst;
    if (all) { st->converged = 1; break; }
    if (its >= c->p.outer_maxiter) { st->converged = 0; break; }
    WCMG_CUDA(cudaMemcpyAsync(mask.p + 1, done.data(), sizeof(int) * nrhs, cudaMemcpyHostToDevice, c->st));
    launch_convert<double, float>(r32, r64, n * nrhs, c->st);
    launch_mask_rhs<float>(r32, mask.p + 1, n, nrhs, c->st);
    KrylovOut k = fgmres<float>(c, 0, e32, r32, nrhs, c->p.outer_restart, inner_tol,
                                std::min(c->p.outer_restart, c->p.outer_maxiter - its), true, false, true, 1);
    its += k.iterations;
    ++restarts;
    if (k.iterations == 0) { st->converged = 0; break; }  // FP32 cycle could not move (no progress)
    launch_convert<float, double>(t64, e32, n * nrhs, c->st);
    launch_axpby<double>(x, 1.0, t64, 1.0, n, nrhs, c->st);
    apply_op<double>(c, 0, t64, x, nrhs);
    copy_fields<double>(c, r64, b, n * nrhs);
    launch_axpby<double>(r64, -1.0, t64, 1.0, n, nrhs, c->st);
  }
  st->outer_iterations = its;
  st->restarts = restarts - 1 > 0 ? restarts - 1 : 0;
  WCMG_CUDA(cudaStreamSynchronize(c->st));
}

// ---------------- the solve as one CUDA graph ----------------
// solve_mixed / solve_f64 with the device-side tests of fgmres_g: captured once per
// (nrhs, buffer generation) and replayed by a single cudaGraphLaunch.

static void solve_mixed_body(wcmg_ctx* c, double2* x, const double2* b, int nrhs) {
  Level& L = c->L[0];
  const long long n = L.n();
  double2* r64 = ws<double>(L, "mx_r", nrhs);
  double2* t64 = ws<double>(L, "mx_t", nrhs);
  float2* r32 = ws<float>(L, "mx_r32", nrhs);
  float2* e32 = ws<float>(L, "mx_e32", nrhs);
  L.sc.ensure(max_rhs_all(c), std::max(c->p.outer_restart, c->p.coarse_restart));
  double* bn2 = L.sc.slot(7);
  KCtl* Kmx = c->kctl.p;
  KCtl* Kfg = c->kctl.p + 1;
  norm2_op<double>(c, bn2, b, n, nrhs);
  start_residual(c, x, r64, t64, b, nrhs);
  norm2_op<double>(c, L.sc.slot(1), r64, n, nrhs);
  const cudaGraphConditionalHandle h = cond_handle(c);
  launch_kctl_init(Kmx, c->p.outer_maxiter, nullptr, 0, h, 0, c->st);
  launch_mx_check(Kmx, nullptr, L.sc.slot(1), bn2, c->p.outer_tol, c->mx_done.p, c->mx_worst.p, nrhs,
                  BodyCount{nullptr, -1, nullptr}, h, c->st);
  cond_node(c, h, cudaGraphCondTypeWhile, [&](int slot) {
    launch_convert<double, float>(r32, r64, n * nrhs, c->st);
    launch_mask_rhs<float>(r32, c->mx_done.p, n, nrhs, c->st);
    fgmres_g<float>(c, 0, e32, r32, nrhs, c->p.outer_restart, kInnerTol, c->p.outer_restart, true, false, true, 1,
                    Kfg, &Kmx->its, c->p.outer_maxiter, nullptr);
    launch_convert<float, double>(t64, e32, n * nrhs, c->st);
    launch_axpby<double>(x, 1.0, t64, 1.0, n, nrhs, c->st);
    apply_op<double>(c, 0, t64, x, nrhs);
    copy_fields<double>(c, r64, b, n * nrhs);
    launch_axpby<double>(r64, -1.0, t64, 1.0, n, nrhs, c->st);
    norm2_op<double>(c, L.sc.slot(1), r64, n, nrhs);
    launch_mx_check(Kmx, Kfg, L.sc.slot(1), bn2, c->p.outer_tol, c->mx_done.p, c->mx_worst.p, nrhs,
                    body_count(c, slot), h, c->st);
  });
}

static void solve_f64_body(wcmg_ctx* c, double2* x, const double2* b, int nrhs) {
  fgmres_g<double>(c, 0, x, b, nrhs, c->p.outer_restart, c->p.outer_tol, c->p.outer_maxiter, !c->guess, true,
                   true, 0, c->kctl.p + 1, nullptr, 0, nullptr);
}

// Device buffers of the graph path and every lazily converted operand, made
// eagerly so that neither a capture nor a replay allocates or converts.
static void graph_prepare(wcmg_ctx* c, int nrhs) {
  c->body_counts.ensure(wcmg_ctx::MAX_BODIES);
  c->gstat.ensure(2);
  c->kctl.ensure(2 + 2 * WCMG_MAX_LEVELS);
  c->mx_done.ensure(max_rhs_all(c));
  c->mx_worst.ensure(1);
  for (auto& s : c->cap_st)
    if (!s) WCMG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  // the basis-slot copies of fgmres_g (level-0 FGMRES, coarsest GMRES, GMRES smoothers)
  const int lc = c->p.n_levels - 1;
  const bool gsm = c->p.smoother == WCMG_SMOOTHER_GMRES;
  if (inner64(c)) {
    ws<double>(c->L[0], "fg_vc", nrhs);
    ws<double>(c->L[0], "fg_zc", nrhs);
    ws<double>(c->L[lc], "gm_vc", nrhs);
    for (int l = 0; gsm && l < lc; ++l) ws<double>(c->L[l], "gm_vc", nrhs);
    for (int l = 1; c->p.kcycle && l < lc; ++l) {
      ws<double>(c->L[l], "fg_vc", nrhs);
      ws<double>(c->L[l], "fg_zc", nrhs);
    }
    return;
  }
  ws<float>(c->L[0], "fg_vc", nrhs);
  ws<float>(c->L[0], "fg_zc", nrhs);
  ws<float>(c->L[lc], "gm_vc", nrhs);
  for (int l = 0; gsm && l < lc; ++l) ws<float>(c->L[l], "gm_vc", nrhs);
  for (int l = 1; c->p.kcycle && l < lc; ++l) {
    ws<float>(c->L[l], "fg_vc", nrhs);
    ws<float>(c->L[l], "fg_zc", nrhs);
  }
  for (int l = 0; l + 1 < c->p.n_levels; ++l) Prec<float>::vecs(c, c->L[l]);
  for (int l = 1; l < c->p.n_levels; ++l) {
    Level& L = c->L[l];
    if (L.have_op && !L.L32_valid && L.op64) {
      const long long n = (long long)L.g.V * L.nc * links_ld(L.nc);
      L.L32.ensure(n);
      launch_convert_links<double2, float2>(L.L32.p, L.L64.p, n, c->st);
      L.L32_valid = true;
      if (c->p.coarse_sigma3 && L.sigma3) build_links5_of<float2>(c, l, L.L32.p);
    }
  }
}

static bool is_warm(const wcmg_ctx* c, int nrhs) {
  return std::find(c->warm_rhs.begin(), c->warm_rhs.end(), nrhs) != c->warm_rhs.end();
}

// Capture the solves of n contexts (each on its own branch) into one graph.
// xs/bs are the contexts' internal FP64 work fields.
static void capture_group(wcmg_ctx** cs, int n, double2* const* xs, const double2* const* bs, const int* nrhs,
                          wcmg_ctx::Graph& G) {
  wcmg_ctx* c0 = cs[0];
  for (int i = 0; i < n; ++i)
    if (!cs[i]->cap_st[0]) WCMG_CUDA(cudaStreamCreateWithFlags(&cs[i]->cap_st[0], cudaStreamNonBlocking));
  cudaStream_t ms = c0->cap_st[0];
  std::vector<cudaStream_t> saved(n);
  for (int i = 0; i < n; ++i) saved[i] = cs[i]->st;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins(n, nullptr);
  WCMG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (int i = 1; i < n; ++i) WCMG_CUDA(cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming));
  auto cleanup = [&]() {
    for (int i = 0; i < n; ++i) {
      cs[i]->st = saved[i];
      cs[i]->capturing = false;
      cs[i]->cap_depth = 0;
      cs[i]->nested.clear();
    }
    cudaEventDestroy(fork);
    for (auto e : joins)
      if (e) cudaEventDestroy(e);
  };
  WCMG_CUDA(cudaStreamBeginCapture(ms, cudaStreamCaptureModeRelaxed));
  cudaGraph_t g = nullptr;
  try {
    WCMG_CUDA(cudaEventRecord(fork, ms));
    for (int i = 0; i < n; ++i) {
      wcmg_ctx* c = cs[i];
      c->st = c->cap_st[0];
      if (i > 0) WCMG_CUDA(cudaStreamWaitEvent(c->st, fork, 0));
      c->capturing = true;
      c->cap_depth = 0;
      c->body_counts_h.clear();
      c->nested.assign(1, 0);
      WCMG_CUDA(cudaMemsetAsync(c->gstat.p, 0, 2 * sizeof(long long), c->st));
      const long long l0 = launch_counter();
      if (inner64(c)) solve_f64_body(c, xs[i], bs[i], nrhs[i]);
      else solve_mixed_body(c, xs[i], bs[i], nrhs[i]);
      c->graph_top = (launch_counter() - l0) - c->nested[0];
      c->capturing = false;
      if (i > 0) {
        WCMG_CUDA(cudaEventRecord(joins[i], c->st));
        WCMG_CUDA(cudaStreamWaitEvent(ms, joins[i], 0));
      }
    }
    WCMG_CUDA(cudaStreamEndCapture(ms, &g));
  } catch (...) {
    cudaGraph_t dummy = nullptr;
    cudaStreamEndCapture(ms, &dummy);
    if (dummy) cudaGraphDestroy(dummy);
    cleanup();
    throw;
  }
  cleanup();
  cudaGraphExec_t exec = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    throw Error(WCMG_ERR_CUDA, std::string("graph instantiation: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < n; ++i) {
    wcmg_ctx* c = cs[i];
    if (!c->body_counts_h.empty())
      WCMG_CUDA(cudaMemcpy(c->body_counts.p, c->body_counts_h.data(), sizeof(int) * c->body_counts_h.size(),
                           cudaMemcpyHostToDevice));
  }
  G.reset();
  G.g = g;
  G.exec = exec;
  G.gen = graph_epoch();
}

// Replay results of one context: iterations, residual, launches.
static void graph_stats(wcmg_ctx* c, wcmg_stats* st) {
  KCtl k[2];
  long long gs[2];
  double worst = 0.0;
  WCMG_CUDA(cudaMemcpyAsync(k, c->kctl.p, sizeof(k), cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaMemcpyAsync(gs, c->gstat.p, sizeof(gs), cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaMemcpyAsync(&worst, c->mx_worst.p, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  if (inner64(c)) {
    if (k[1].err) throw Error(WCMG_ERR_NAN, "non-finite residual in Krylov solver");
    st->outer_iterations = k[1].its;
    st->restarts = k[1].cycles > 1 ? k[1].cycles - 1 : 0;
  } else {
    if (k[0].err) throw Error(WCMG_ERR_NAN, "non-finite residual");
    st->outer_iterations = k[0].its;
    st->restarts = k[0].restarts - 1 > 0 ? k[0].restarts - 1 : 0;
    st->true_residual = worst;
  }
  st->coarse_iterations = gs[1];
  st->kernel_launches = c->graph_top + gs[0];
  st->graph = 1;
}

// true residual max_r ||b - D x|| / ||b|| in FP64
static double true_residual(wcmg_ctx* c, const double2* x, const double2* b, int nrhs) {
  Level& L = c->L[0];
  const long long n = L.n();
  double2* t = ws<double>(L, "tr_t", nrhs);
  apply_op<double>(c, 0, t, x, nrhs);
  launch_axpby<double>(t, 1.0, b, -1.0, n, nrhs, c->st);
  L.sc.ensure(max_rhs_all(c), std::max(c->p.outer_restart, c->p.coarse_restart));
  norm2_op<double>(c, L.sc.slot(1), t, n, nrhs);
  norm2_op<double>(c, L.sc.slot(7), b, n, nrhs);
  std::vector<double> rn(nrhs);
  const double* h = read_doubles(c, L.sc.slot(1), nrhs);
  for (int q = 0; q < nrhs; ++q) rn[q] = h[q];
  h = read_doubles(c, L.sc.slot(7), nrhs);
  double worst = 0;
  for (int q = 0; q < nrhs; ++q) worst = std::max(worst, h[q] > 0 ? std::sqrt(rn[q] / h[q]) : 0.0);
  return worst;
}

// ---------------- training of the learned coarse correction ----------------
// Pairs (r, e = P GMRES(D_c; P^dag r)) are generated with the current hierarchy
// in FP32 batches: half Gaussian r, half residuals r = b - D M_0(b) of one
// multigrid cycle on a Gaussian b (the kind of vectors FGMRES feeds its
// preconditioner); each r is normalised.  The loss is the mean over pairs of
// ||N(r) - e||^2 / ||e||^2; Adam steps over contiguous minibatches.
static double ptc_eval(wcmg_ctx* c, int npairs, int chunk) {
  Level& L = c->L[0];
  const long long n = L.n();
  float2* out = ws<float>(L, "ptc_out", chunk);
  double total = 0.0;
  for (int p0 = 0; p0 < npairs; p0 += chunk) {
    const int k = std::min(chunk, npairs - p0);
    ptc_forward(c, out, c->ds_r.p + p0 * n, k);
    launch_axpby<float>(out, -1.0, c->ds_e.p + p0 * n, 1.0, n, k, c->st);  // out = N(r) - e
    norm2_op<float>(c, L.sc.slot(7), out, n, k);
    norm2_op<float>(c, L.sc.slot(6), c->ds_e.p + p0 * n, n, k);
    std::vector<double> d2(k);
    const double* h = read_doubles(c, L.sc.slot(7), k);
    for (int q = 0; q < k; ++q) d2[q] = h[q];
    h = read_doubles(c, L.sc.slot(6), k);
    for (int q = 0; q < k; ++q) total += d2[q] / h[q];
  }
  return total / npairs;
}

static void ptc_train(wcmg_ctx* c, const wcmg_train_opts* o, wcmg_train_stats* st) {
  if (c->p.inner_prec != WCMG_F32) throw Error(WCMG_ERR_ARG, "training needs inner_prec F32");
  for (int l = 0; l + 1 < c->p.n_levels; ++l)
    if (!c->L[l].have_P || !c->L[l + 1].have_op) throw Error(WCMG_ERR_STATE, "setup not done");
  const int np = o->npairs, B = o->batch;
  const int chunk = max_rhs_all(c);
  if (np < 1 || B < 1 || B > chunk || o->steps < 0 || o->refresh < 0)
    throw Error(WCMG_ERR_ARG, "npairs/batch/steps/refresh out of range");
  Level& L = c->L[0];
  Level& C1 = c->L[1];
  const long long n = L.n();
  L.sc.ensure(chunk, std::max(c->p.outer_restart, c->p.coarse_restart));
  ptc_alloc(c);
  if (!c->have_ptc) {  // small random start (counter-based generator), the scale keeps N(r) ~ 0.05 r
    launch_gaussian_field(c->ptcW.p, WCMG_PTC_NWEIGHTS, o->seed, 977, c->st);
    launch_axpby<float>(c->ptcW.p, 0.0, c->ptcW.p, 0.02, WCMG_PTC_NWEIGHTS, 1, c->st);
    c->have_ptc = true;
  }
  WCMG_CUDA(cudaMemsetAsync(c->ptcM.p, 0, sizeof(float2) * WCMG_PTC_NWEIGHTS, c->st));
  WCMG_CUDA(cudaMemsetAsync(c->ptcV.p, 0, sizeof(float2) * WCMG_PTC_NWEIGHTS, c->st));
  c->ptc_t = 0;
  c->ds_r.ensure((size_t)np * n);
  c->ds_e.ensure((size_t)np * n);
  c->ptcScale.ensure(np);
  const bool saved_on = c->learned_on;
  c->learned_on = false;
  double ms_gen = 0.0;
  long long pools = 0;
  // a pool of np pairs from generator stream `pool` (every pool draws fresh fields)
  auto generate = [&](long long pool) {
    WCMG_CUDA(cudaStreamSynchronize(c->st));  // queued training steps count as training time
    auto g0 = std::chrono::steady_clock::now();
    for (int p0 = 0; p0 < np; p0 += chunk) {
      const int k = std::min(chunk, np - p0);
      float2* r = c->ds_r.p + p0 * n;
      float2* e = c->ds_e.p + p0 * n;
      launch_gaussian_field(r, (long long)k * n, o->seed, 1 + p0 + (unsigned long long)pool * 1000003ULL, c->st);
      const int nh = k / 2;  // the second half becomes residuals after one cycle
      if (nh > 0) {
        float2* b = r + (k - nh) * n;
        float2* x = ws<float>(L, "ptc_x", nh);
        float2* t = ws<float>(L, "ptc_t", nh);
        cycle<float>(c, 0, x, b, nh);
        apply_op<float>(c, 0, t, x, nh);
        launch_axpby<float>(b, -1.0, t, 1.0, n, nh, c->st);  // b <- b - D M(b)
      }
      norm2_op<float>(c, L.sc.slot(7), r, n, k);
      launch_scale_dev<float>(r, r, L.sc.slot(7), 1, n, k, c->st);
      float2* rc = ws<float>(C1, "ptc_rc", k);
      float2* ec = ws<float>(C1, "ptc_ec", k);
      restrict_op<float>(c, 0, rc, r, k);
      if (c->p.n_levels == 2) {
        fgmres<float>(c, 1, ec, rc, k, c->p.coarse_restart, o->target_tol, 2000, true, false, false);
      } else {
        cycle<float>(c, 1, ec, rc, k);  // deeper hierarchies: one coarse cycle as the target
      }
      prolong_op<float>(c, 0, e, ec, k);
    }
    // per-pair gradient scale 1 / (||e||^2 B)
    std::vector<double> sc(np);
    for (int p0 = 0; p0 < np; p0 += chunk) {
      const int k = std::min(chunk, np - p0);
      norm2_op<float>(c, L.sc.slot(6), c->ds_e.p + p0 * n, n, k);
      const double* h = read_doubles(c, L.sc.slot(6), k);
      for (int q = 0; q < k; ++q) sc[p0 + q] = 1.0 / (h[q] * B);
    }
    WCMG_CUDA(cudaMemcpyAsync(c->ptcScale.p, sc.data(), sizeof(double) * np, cudaMemcpyHostToDevice, c->st));
    WCMG_CUDA(cudaStreamSynchronize(c->st));
    ms_gen += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g0).count();
    ++pools;
  };
  generate(0);
  st->loss_initial = ptc_eval(c, np, chunk);
  auto t1 = std::chrono::steady_clock::now();
  const double gen_before = ms_gen;
  float2* out = ws<float>(L, "ptc_out", chunk);
  int pool_step = 0;
  for (int step = 0; step < o->steps; ++step) {
    if (o->refresh > 0 && step > 0 && step % o->refresh == 0) {
      generate(pools);
      pool_step = 0;
    }
    const int p0 = (int)(((long long)pool_step * B) % np);
    ++pool_step;
    const int k = std::min(B, np - p0);
    const float2* rb = c->ds_r.p + p0 * n;
    ptc_forward(c, out, rb, k);
    launch_axpby<float>(out, -1.0, c->ds_e.p + p0 * n, 1.0, n, k, c->st);       // N(r) - e
    launch_scale_dev<float>(out, out, c->ptcScale.p + p0, 0, n, k, c->st);      // dL/d conj(N)
    ptc_backward(c, rb, out, nullptr, k);
    ++c->ptc_t;
    KPROF(c, WCMG_K_PTC, 5.0 * WCMG_PTC_NWEIGHTS * 8, 0.0,
          launch_ptc_adam(c->ptcW.p, c->ptcG.p, c->ptcM.p, c->ptcV.p, WCMG_PTC_NWEIGHTS, (float)o->lr, c->ptc_t,
                          c->st));
  }
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  auto t2 = std::chrono::steady_clock::now();
  const double gen_in_loop = ms_gen - gen_before;
  st->loss_final = ptc_eval(c, np, chunk);
  st->pairs_total = pools * (long long)np;
  generate(pools);  // held out: never trained on
  st->loss_heldout = ptc_eval(c, np, chunk);
  st->ms_generate = ms_gen;
  st->ms_train = std::chrono::duration<double, std::milli>(t2 - t1).count() - gen_in_loop;
  c->learned_on = saved_on;
}

// FP32 copy of the clover term and, for the even-odd SAP smoother, C^-1 (FP64 and
// FP32), after clover64 changed.
static void clover_derived(wcmg_ctx* c) {
  const int V = c->L[0].g.V;
  launch_convert<double, float>(c->clover32.p, c->clover64.p, (long long)36 * V, c->st);
  if (c->p.sap_eo) {
    c->cinv64.ensure((size_t)36 * V);
    c->cinv32.ensure((size_t)36 * V);
    c->cinv_err.ensure(1);
    WCMG_CUDA(cudaMemsetAsync(c->cinv_err.p, 0, sizeof(int), c->st));
    KPROF(c, WCMG_K_CLOVER, 36.0 * V * 16 * 2, 2.0 * V * 6 * 6 * 12 * 8,
          launch_clover_invert(c->cinv64.p, c->clover64.p, V, c->cinv_err.p, c->st));
    launch_convert<double, float>(c->cinv32.p, c->cinv64.p, (long long)36 * V, c->st);
    int bad = 0;
    WCMG_CUDA(cudaMemcpyAsync(&bad, c->cinv_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WCMG_CUDA(cudaStreamSynchronize(c->st));
    if (bad) throw Error(WCMG_ERR_NAN, "singular clover block: no even-odd SAP");
  }
}

// ---------------- external I/O ----------------
static const double2* in_dev(wcmg_ctx* c, const void* ptr, size_t bytes, int where, int slot) {
  if (where == WCMG_DEVICE) return (const double2*)ptr;
  if (where != WCMG_HOST) throw Error(WCMG_ERR_ARG, "where must be WCMG_HOST or WCMG_DEVICE");
  auto* d = c->stage[slot].ensure(bytes);
  WCMG_CUDA(cudaMemcpyAsync(d, ptr, bytes, cudaMemcpyHostToDevice, c->st));
  return (const double2*)d;
}
static double2* out_dev(wcmg_ctx* c, void* ptr, size_t bytes, int where, int slot) {
  if (where == WCMG_DEVICE) return (double2*)ptr;
  if (where != WCMG_HOST) throw Error(WCMG_ERR_ARG, "where must be WCMG_HOST or WCMG_DEVICE");
  return (double2*)c->stage[slot].ensure(bytes);
}
static void out_finish(wcmg_ctx* c, void* ptr, const double2* d, size_t bytes, int where) {
  if (where == WCMG_HOST) {
    WCMG_CUDA(cudaMemcpyAsync(ptr, d, bytes, cudaMemcpyDeviceToHost, c->st));
    WCMG_CUDA(cudaStreamSynchronize(c->st));
  }
}

template <typename R>
static void pack_level(wcmg_ctx* c, int l, cplx<R>* out, const double2* ext, int nrhs) {
  Level& L = c->L[l];
  KPROF(c, WCMG_K_PACK, (double)L.n() * nrhs * (16.0 + sizeof(cplx<R>)), 0.0,
        (L.fine ? launch_pack_fine<R>(out, ext, L.g.d_perm.p, L.g.V, nrhs, c->st)
                : launch_pack_coarse<R>(out, ext, L.g.d_perm.p, L.g.V, L.nc, nrhs, c->st)));
}
template <typename R>
static void unpack_level(wcmg_ctx* c, int l, double2* ext, const cplx<R>* in, int nrhs) {
  Level& L = c->L[l];
  KPROF(c, WCMG_K_PACK, (double)L.n() * nrhs * (16.0 + sizeof(cplx<R>)), 0.0,
        (L.fine ? launch_unpack_fine<R>(ext, in, L.g.d_perm.p, L.g.V, nrhs, c->st)
                : launch_unpack_coarse<R>(ext, in, L.g.d_perm.p, L.g.V, L.nc, nrhs, c->st)));
}


// A bounded device-side wait that gave up leaves a nonzero word: report it.
static void check_device_waits(wcmg_ctx* c) {
  const int* e = read_ints(c, c->tma_err.p, 1);
  if (e[0]) {
    WCMG_CUDA(cudaMemsetAsync(c->tma_err.p, 0, sizeof(int), c->st));
    throw Error(WCMG_ERR_TIMEOUT, "a bounded device-side wait gave up");
  }
}

static void kstat_delta(wcmg_kstat* out, const wcmg_kstat* now, const wcmg_kstat* before) {
  for (int i = 0; i < WCMG_NKCLASS; ++i) {
    out[i].launches = now[i].launches - before[i].launches;
    out[i].ms = now[i].ms - before[i].ms;
    out[i].bytes = now[i].bytes - before[i].bytes;
    out[i].flops = now[i].flops - before[i].flops;
  }
}

static void check_level(const wcmg_ctx* c, int l, int lo, int hi) {
  if (l < lo || l > hi) throw Error(WCMG_ERR_ARG, "level out of range");
  (void)c;
}
static void check_rhs(const wcmg_ctx* c, int nrhs) {
  if (nrhs < 1 || nrhs > max_rhs_all(c)) throw Error(WCMG_ERR_ARG, "nrhs out of range (1 .. max_rhs)");
}

}  // namespace wcmg

// =====================================================================
// C-ABI
// =====================================================================
#define API_BEGIN(ctx)                    \
  if (!(ctx)) return WCMG_ERR_ARG;        \
  try {
#define API_END(ctx)                                                     \
  }                                                                      \
  catch (const wcmg::Error& e) {                                         \
    (ctx)->err = e.what();                                               \
    (ctx)->prof.pend.clear();                                            \
    return e.code;                                                       \
  }                                                                      \
  catch (const std::exception& e) {                                      \
    (ctx)->err = e.what();                                               \
    return WCMG_ERR_ARG;                                                 \
  }                                                                      \
  return WCMG_OK;

extern "C" {

int wcmg_default_params(wcmg_params* p) {
  if (!p) return WCMG_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  for (int k = 0; k < 4; ++k) p->dims[k] = 4;
  p->n_levels = 2;
  for (int l = 0; l < WCMG_MAX_LEVELS - 1; ++l) {
    for (int k = 0; k < 4; ++k) p->block[l][k] = 2;
    p->nvec[l] = 8;
  }
  p->m0 = -0.1;
  p->csw = 1.0;
  p->smoother_steps = 4;
  p->setup_init_sweeps = 3;
  p->setup_refine_sweeps = 0;
  p->coarse_restart = 20;
  p->coarse_maxiter = 100;
  p->coarse_tol = 0.05;
  p->outer_restart = 20;
  p->outer_maxiter = 1000;
  p->outer_tol = 1e-10;
  p->inner_prec = WCMG_F64;
  p->coarse_link_prec = WCMG_F32;
  p->max_rhs = 1;
  p->profile = 0;
  p->use_graphs = 0;
  p->autotune = 0;
  p->smoother = WCMG_SMOOTHER_MR;
  p->kcycle = 0;
  p->kcycle_steps = 5;
  p->kcycle_tol = 0.1;
  p->sap_cycles = 1;
  p->sap_eo = 0;
  p->ortho_df = 0;
  p->coarse_eo = 0;
  p->coarse_sigma3 = 0;
  return WCMG_OK;
}

int wcmg_create(const wcmg_params* p, wcmg_ctx** out) {
  if (!p || !out) return WCMG_ERR_ARG;
  *out = nullptr;
  wcmg_ctx* c = new (std::nothrow) wcmg_ctx();
  if (!c) return WCMG_ERR_OOM;
  c->p = *p;
  try {
    const int nl = p->n_levels;
    if (nl < 2 || nl > WCMG_MAX_LEVELS) throw Error(WCMG_ERR_ARG, "n_levels must be 2..4");
    if (p->inner_prec != WCMG_F64 && p->inner_prec != WCMG_F32) throw Error(WCMG_ERR_ARG, "inner_prec");
    if (p->coarse_link_prec != WCMG_F32 && p->coarse_link_prec != WCMG_BF16 && p->coarse_link_prec != WCMG_F16 &&
        p->coarse_link_prec != WCMG_F64)
      throw Error(WCMG_ERR_ARG, "coarse_link_prec");
    if (p->smoother_steps < 0 || p->coarse_restart < 1 || p->outer_restart < 1 || p->coarse_restart > 64 ||
        p->outer_restart > 64 || p->max_rhs < 1 || p->max_rhs > 1024)
      throw Error(WCMG_ERR_ARG, "solver parameters out of range");
    if ((p->use_graphs != 0 && p->use_graphs != 1) || (p->autotune != 0 && p->autotune != 1))
      throw Error(WCMG_ERR_ARG, "use_graphs and autotune must be 0 or 1");
    if (p->smoother != WCMG_SMOOTHER_MR && p->smoother != WCMG_SMOOTHER_GMRES && p->smoother != WCMG_SMOOTHER_SAP)
      throw Error(WCMG_ERR_ARG, "smoother must be WCMG_SMOOTHER_MR, WCMG_SMOOTHER_GMRES or WCMG_SMOOTHER_SAP");
    if (p->sap_cycles < 1 || p->sap_cycles > 16) throw Error(WCMG_ERR_ARG, "sap_cycles must be 1..16");
    if (p->sap_eo != 0 && p->sap_eo != 1) throw Error(WCMG_ERR_ARG, "sap_eo must be 0 or 1");
    if (p->ortho_df != 0 && p->ortho_df != 1) throw Error(WCMG_ERR_ARG, "ortho_df must be 0 or 1");
    if (p->coarse_eo != 0 && p->coarse_eo != 1) throw Error(WCMG_ERR_ARG, "coarse_eo must be 0 or 1");
    if (p->coarse_sigma3 != 0 && p->coarse_sigma3 != 1) throw Error(WCMG_ERR_ARG, "coarse_sigma3 must be 0 or 1");
    if (p->sap_eo) {
      const int* fb = p->block[0];
      const int bv = fb[0] * fb[1] * fb[2] * fb[3];
      if ((fb[0] & 1) || bv > 256)
        throw Error(WCMG_ERR_ARG, "sap_eo needs fine aggregates of at most 256 sites with an even x extent");
    }
    if (p->smoother_steps > 64) throw Error(WCMG_ERR_ARG, "smoother_steps: at most 64");
    if ((p->kcycle != 0 && p->kcycle != 1) || p->kcycle_steps < 1 || p->kcycle_steps > 64 || !(p->kcycle_tol >= 0.0))
      throw Error(WCMG_ERR_ARG, "kcycle must be 0 or 1, kcycle_steps 1..64, kcycle_tol >= 0");
    c->L.resize(nl);
    int dims[4];
    for (int k = 0; k < 4; ++k) dims[k] = p->dims[k];
    for (int l = 0; l < nl; ++l) {
      Level& L = c->L[l];
      for (int k = 0; k < 4; ++k) {
        if (dims[k] < 1) throw Error(WCMG_ERR_ARG, "lattice extent < 1");
        L.g.dims[k] = dims[k];
      }
      L.g.V = dims[0] * dims[1] * dims[2] * dims[3];
      L.fine = l == 0;
      L.nc = l == 0 ? 12 : 2 * p->nvec[l - 1];
      if (l + 1 < nl) {
        L.nvec = p->nvec[l];
        if (L.nvec < 1 || L.nvec > 32) throw Error(WCMG_ERR_ARG, "nvec must be 1..32");
        for (int k = 0; k < 4; ++k) {
          const int b = p->block[l][k];
          if (b < 1 || dims[k] % b) throw Error(WCMG_ERR_ARG, "extent not divisible by block");
          L.g.b[k] = b;
          dims[k] /= b;
        }
        L.g.bvol = L.g.b[0] * L.g.b[1] * L.g.b[2] * L.g.b[3];
        if (L.g.bvol * (L.nc / 2) < L.nvec) throw Error(WCMG_ERR_ARG, "aggregate too small for nvec (rank)");
        if (L.g.bvol * (L.nc / 2) > 2048) throw Error(WCMG_ERR_ARG, "aggregate panel larger than 2048 rows");
      }
    }
    if (p->coarse_eo) {
      const HostGeom& Gc = c->L[nl - 1].g;
      for (int k = 0; k < 4; ++k)
        if (Gc.dims[k] % 2) throw Error(WCMG_ERR_ARG, "coarse_eo needs even extents of the coarsest lattice");
    }
    // storage orders, coarsest first
    for (int l = nl - 1; l >= 0; --l) {
      HostGeom& G = c->L[l].g;
      G.perm.assign(G.V, 0);
      G.inv.assign(G.V, 0);
      for (int s = 0; s < G.V; ++s) {
        int x[4];
        coords(s, G.dims, x);
        int stg;
        if (l == nl - 1) {
          stg = s;
        } else {
          const HostGeom& Cg = c->L[l + 1].g;
          int xc[4], lo[4];
          for (int k = 0; k < 4; ++k) { xc[k] = x[k] / G.b[k]; lo[k] = x[k] % G.b[k]; }
          stg = Cg.inv[lexi(xc, Cg.dims)] * G.bvol + lexi(lo, G.b);
        }
        G.inv[s] = stg;
        G.perm[stg] = s;
      }
      G.nbr.assign((size_t)8 * G.V, 0);
      for (int st = 0; st < G.V; ++st) {
        int x[4];
        coords(G.perm[st], G.dims, x);
        for (int mu = 0; mu < 4; ++mu)
          for (int dir = 0; dir < 2; ++dir) {
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[mu] = (y[mu] + (dir == 0 ? 1 : G.dims[mu] - 1)) % G.dims[mu];
            G.nbr[(size_t)(2 * mu + dir) * G.V + st] = G.inv[lexi(y, G.dims)];
          }
      }
      G.d_perm.ensure(G.V);
      G.d_nbr.ensure((size_t)8 * G.V);
      {
        std::vector<unsigned char> par(G.V);
        for (int st = 0; st < G.V; ++st) {
          int x[4];
          coords(G.perm[st], G.dims, x);
          par[st] = (unsigned char)((x[0] + x[1] + x[2] + x[3]) & 1);
        }
        G.d_par.ensure(G.V);
        WCMG_CUDA(cudaMemcpy(G.d_par.p, par.data(), G.V, cudaMemcpyHostToDevice));
      }
      WCMG_CUDA(cudaMemcpy(G.d_perm.p, G.perm.data(), sizeof(int) * G.V, cudaMemcpyHostToDevice));
      WCMG_CUDA(cudaMemcpy(G.d_nbr.p, G.nbr.data(), sizeof(int) * 8 * G.V, cudaMemcpyHostToDevice));
      if (l + 1 < nl) {
        // SAP colours: aggregate B of this level is site B of the next level's storage
        const HostGeom& Cg = c->L[l + 1].g;
        std::vector<unsigned char> col(Cg.V);
        for (int B = 0; B < Cg.V; ++B) {
          int xc[4];
          coords(Cg.perm[B], Cg.dims, xc);
          col[B] = (unsigned char)((xc[0] + xc[1] + xc[2] + xc[3]) & 1);
        }
        std::vector<int> list;
        for (int k = 0; k < 2; ++k)
          for (int B = 0; B < Cg.V; ++B)
            if (col[B] == k) list.push_back(B);
        Level& Lc = c->L[l];
        std::vector<unsigned char> op(Cg.V);
        for (int B = 0; B < Cg.V; ++B) {
          int xc[4];
          coords(Cg.perm[B], Cg.dims, xc);
          int par = 0;
          for (int k = 0; k < 4; ++k) par += xc[k] * G.b[k];
          op[B] = (unsigned char)(par & 1);
        }
        Lc.opar.ensure(Cg.V);
        WCMG_CUDA(cudaMemcpy(Lc.opar.p, op.data(), Cg.V, cudaMemcpyHostToDevice));
        Lc.sap_count[0] = (int)std::count(col.begin(), col.end(), 0);
        Lc.sap_count[1] = Cg.V - Lc.sap_count[0];
        Lc.colour.ensure(Cg.V);
        Lc.sap_list.ensure(Cg.V);
        WCMG_CUDA(cudaMemcpy(Lc.colour.p, col.data(), Cg.V, cudaMemcpyHostToDevice));
        WCMG_CUDA(cudaMemcpy(Lc.sap_list.p, list.data(), sizeof(int) * Cg.V, cudaMemcpyHostToDevice));
      }
    }
    ensure_partials(c);
    for (auto& L : c->L) L.sc.ensure(max_rhs_all(c), std::max(c->p.outer_restart, c->p.coarse_restart));
    c->errflag.ensure((size_t)max_rhs_all(c) + 1);
    c->tma_err.ensure(1);
    WCMG_CUDA(cudaMemset(c->tma_err.p, 0, sizeof(int)));
    c->prof.mask = p->profile;
  } catch (const Error& e) {
    int code = e.code;
    delete c;
    return code;
  }
  *out = c;
  return WCMG_OK;
}

void wcmg_destroy(wcmg_ctx* ctx) { delete ctx; }

const char* wcmg_last_error(const wcmg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int wcmg_set_gauge(wcmg_ctx* c, const void* U, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  Level& L = c->L[0];
  const int V = L.g.V;
  const double2* u = in_dev(c, U, (size_t)4 * V * 9 * 16, where, 0);
  c->gauge64.ensure((size_t)36 * V);
  c->gauge32.ensure((size_t)36 * V);
  c->clover64.ensure((size_t)36 * V);
  c->clover32.ensure((size_t)36 * V);
  KPROF(c, WCMG_K_PACK, 36.0 * V * 32, 0, launch_pack_gauge<double>(c->gauge64.p, u, L.g.d_perm.p, V, c->st));
  launch_pack_gauge<float>(c->gauge32.p, u, L.g.d_perm.p, V, c->st);
  KPROF(c, WCMG_K_CLOVER, 36.0 * V * 16 * 5, 0,
        launch_clover_build(c->clover64.p, c->gauge64.p, L.g.d_nbr.p, V, c->p.m0, c->p.csw, c->st));
  clover_derived(c);
  c->have_gauge = true;
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  c->prof.flush();
  API_END(c)
}

int wcmg_set_clover(wcmg_ctx* c, double csw, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  if (!std::isfinite(csw)) throw Error(WCMG_ERR_ARG, "csw must be finite");
  c->p.csw = csw;
  Level& L = c->L[0];
  const int V = L.g.V;
  KPROF(c, WCMG_K_CLOVER, 36.0 * V * 16 * 5, 0,
        launch_clover_build(c->clover64.p, c->gauge64.p, L.g.d_nbr.p, V, c->p.m0, c->p.csw, c->st));
  clover_derived(c);
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  c->prof.flush();
  API_END(c)
}

int wcmg_set_clover_raw(wcmg_ctx* c, const void* C, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  if (!C) throw Error(WCMG_ERR_ARG, "null clover");
  Level& L = c->L[0];
  const int V = L.g.V;
  const double2* e = in_dev(c, C, (size_t)V * 144 * 16, where, 0);
  c->cinv_err.ensure(1);
  WCMG_CUDA(cudaMemsetAsync(c->cinv_err.p, 0, sizeof(int), c->st));
  DevBuf<double2> packed;  // the context's clover stays untouched if the blocks are rejected
  packed.ensure((size_t)36 * V);
  KPROF(c, WCMG_K_CLOVER, (double)V * (144 + 36) * 16, 0,
        launch_clover_pack(packed.p, e, L.g.d_perm.p, V, 1e-12, c->cinv_err.p, c->st));
  int bad = 0;
  WCMG_CUDA(cudaMemcpyAsync(&bad, c->cinv_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  if (bad) throw Error(WCMG_ERR_ARG, "clover blocks must be Hermitian and block diagonal in chirality");
  WCMG_CUDA(cudaMemcpyAsync(c->clover64.p, packed.p, sizeof(double2) * 36 * V, cudaMemcpyDeviceToDevice, c->st));
  clover_derived(c);
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  c->prof.flush();
  API_END(c)
}

int wcmg_get_clover(wcmg_ctx* c, void* C, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  const int V = c->L[0].g.V;
  const size_t bytes = (size_t)V * 144 * 16;
  double2* o = out_dev(c, C, bytes, where, 1);
  launch_clover_expand(o, c->clover64.p, c->L[0].g.d_perm.p, V, c->st);
  out_finish(c, C, o, bytes, where);
  API_END(c)
}

int wcmg_get_clover_inverse(wcmg_ctx* c, void* C, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  if (!c->cinv64.p) throw Error(WCMG_ERR_STATE, "the inverse clover term is built only with params.sap_eo");
  const int V = c->L[0].g.V;
  const size_t bytes = (size_t)V * 144 * 16;
  double2* o = out_dev(c, C, bytes, where, 1);
  launch_clover_expand(o, c->cinv64.p, c->L[0].g.d_perm.p, V, c->st);
  out_finish(c, C, o, bytes, where);
  API_END(c)
}

extern "C++" {
template <typename R>
static void apply_D_ext(wcmg_ctx* c, const double2* in, double2* out, int nrhs) {
  Level& L = c->L[0];
  cplx<R>* a = ws<R>(L, "io_a", nrhs);
  cplx<R>* b = ws<R>(L, "io_b", nrhs);
  pack_level<R>(c, 0, a, in, nrhs);
  apply_op<R>(c, 0, b, a, nrhs);
  unpack_level<R>(c, 0, out, b, nrhs);
}
}  // extern "C++"

int wcmg_apply_D(wcmg_ctx* c, const void* in, void* out, int nrhs, int prec, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_rhs(c, nrhs);
  const size_t bytes = (size_t)nrhs * c->L[0].n() * 16;
  const double2* i = in_dev(c, in, bytes, where, 0);
  double2* o = out_dev(c, out, bytes, where, 1);
  if (prec == WCMG_F64) apply_D_ext<double>(c, i, o, nrhs);
  else if (prec == WCMG_F32) apply_D_ext<float>(c, i, o, nrhs);
  else throw Error(WCMG_ERR_ARG, "prec must be F64 or F32");
  out_finish(c, out, o, bytes, where);
  API_END(c)
}

int wcmg_set_nullvecs(wcmg_ctx* c, int level, const void* vecs, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 2);
  Level& L = c->L[level];
  const size_t bytes = (size_t)L.nvec * L.n() * 16;
  const double2* v = in_dev(c, vecs, bytes, where, 0);
  if (inner64(c)) {
    L.raw64.ensure((size_t)L.nvec * L.n());
    pack_level<double>(c, level, L.raw64.p, v, L.nvec);
    build_P<double>(c, level);
  } else {
    L.raw32.ensure((size_t)L.nvec * L.n());
    L.raw64.ensure((size_t)L.nvec * L.n());
    pack_level<double>(c, level, L.raw64.p, v, L.nvec);
    // orthonormalise from the FP64 input directly
    L.v64.ensure((size_t)L.nvec * L.n());
    copy_fields<double>(c, L.v64.p, L.raw64.p, (long long)L.nvec * L.n());
    ortho_level(c, level);
    launch_convert<double, float>(L.raw32.p, L.raw64.p, (long long)L.nvec * L.n(), c->st);
    L.v32_valid = false;
    L.have_P = true;
  }
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  c->prof.flush();
  API_END(c)
}

int wcmg_get_nullvecs(wcmg_ctx* c, int level, void* vecs, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 2);
  Level& L = c->L[level];
  if (!L.have_P) throw Error(WCMG_ERR_STATE, "prolongator of level not built");
  const size_t bytes = (size_t)L.nvec * L.n() * 16;
  double2* o = out_dev(c, vecs, bytes, where, 1);
  unpack_level<double>(c, level, o, L.v64.p, L.nvec);
  out_finish(c, vecs, o, bytes, where);
  API_END(c)
}

int wcmg_coarsen(wcmg_ctx* c, int level, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 2);
  if (inner64(c)) coarsen<double>(c, level);
  else coarsen<float>(c, level);
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  c->prof.flush();
  API_END(c)
}

int wcmg_get_coarse_links(wcmg_ctx* c, int level, void* A, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 1, c->p.n_levels - 1);
  Level& L = c->L[level];
  if (!L.have_op) throw Error(WCMG_ERR_STATE, "coarse operator of level not built");
  const int nb = L.nc;
  const size_t bytes = (size_t)9 * L.g.V * nb * nb * 16;
  double2* o = out_dev(c, A, bytes, where, 1);
  if (L.op64) launch_unpack_links<double2>(o, L.L64.p, L.g.d_perm.p, L.g.V, nb, c->st);
  else if (L.L32_valid) launch_unpack_links<float2>(o, L.L32.p, L.g.d_perm.p, L.g.V, nb, c->st);
  else if (L.low_valid && c->p.coarse_link_prec == WCMG_BF16)
    launch_unpack_links<bf16c>(o, L.Lbf.p, L.g.d_perm.p, L.g.V, nb, c->st);
  else if (L.low_valid && c->p.coarse_link_prec == WCMG_F16)
    launch_unpack_links<f16c>(o, L.Lh.p, L.g.d_perm.p, L.g.V, nb, c->st);
  else launch_unpack_links<float2>(o, L.L32.p, L.g.d_perm.p, L.g.V, nb, c->st);
  out_finish(c, A, o, bytes, where);
  API_END(c)
}

int wcmg_set_coarse_links(wcmg_ctx* c, int level, const void* A, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 1, c->p.n_levels - 1);
  Level& L = c->L[level];
  const int nb = L.nc;
  const size_t bytes = (size_t)9 * L.g.V * nb * nb * 16;
  const double2* a = in_dev(c, A, bytes, where, 0);
  const long long nl = (long long)L.g.V * nb * links_ld(nb);
  L.L64.ensure(nl);
  launch_pack_links<double2>(L.L64.p, a, L.g.d_perm.p, L.g.V, nb, c->st);
  L.op64 = true;
  L.L32_valid = false;
  L.low_valid = false;
  if (!inner64(c)) {
    L.L32.ensure(nl);
    launch_convert_links<double2, float2>(L.L32.p, L.L64.p, nl, c->st);
    L.L32_valid = true;
    if (c->p.coarse_link_prec == WCMG_BF16) {
      L.Lbf.ensure(nl);
      launch_convert_links<double2, bf16c>(L.Lbf.p, L.L64.p, nl, c->st);
      build_mma_links(c, level);
      L.low_valid = true;
    } else if (c->p.coarse_link_prec == WCMG_F16) {
      L.Lh.ensure(nl);
      launch_convert_links<double2, f16c>(L.Lh.p, L.L64.p, nl, c->st);
      L.low_valid = true;
    }
  }
  L.have_op = true;
  L.ainv_valid = false;
  L.sigma3 = false;  // caller's blocks: no symmetry assumed, nine-block kernels only
  build_links5(c, level);
  if (c->p.coarse_eo && level == c->p.n_levels - 1) ensure_ainv(c, level);
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  API_END(c)
}

extern "C++" {
template <typename R>
static void transfer_ext(wcmg_ctx* c, int level, const double2* in, double2* out, int nrhs, bool restrict_dir) {
  Level& F = c->L[level];
  Level& C = c->L[level + 1];
  cplx<R>* f = ws<R>(F, "io_a", nrhs);
  cplx<R>* q = ws<R>(C, "io_a", nrhs);
  if (restrict_dir) {
    pack_level<R>(c, level, f, in, nrhs);
    restrict_op<R>(c, level, q, f, nrhs);
    unpack_level<R>(c, level + 1, out, q, nrhs);
  } else {
    pack_level<R>(c, level + 1, q, in, nrhs);
    prolong_op<R>(c, level, f, q, nrhs);
    unpack_level<R>(c, level, out, f, nrhs);
  }
}
}  // extern "C++"

int wcmg_restrict(wcmg_ctx* c, int level, const void* fine, void* coarse, int nrhs, int prec, int where,
                  void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 2);
  check_rhs(c, nrhs);
  const size_t bi = (size_t)nrhs * c->L[level].n() * 16, bo = (size_t)nrhs * c->L[level + 1].n() * 16;
  const double2* i = in_dev(c, fine, bi, where, 0);
  double2* o = out_dev(c, coarse, bo, where, 1);
  if (prec == WCMG_F64) transfer_ext<double>(c, level, i, o, nrhs, true);
  else if (prec == WCMG_F32) transfer_ext<float>(c, level, i, o, nrhs, true);
  else throw Error(WCMG_ERR_ARG, "prec must be F64 or F32");
  out_finish(c, coarse, o, bo, where);
  API_END(c)
}

int wcmg_prolong(wcmg_ctx* c, int level, const void* coarse, void* fine, int nrhs, int prec, int where,
                 void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 2);
  check_rhs(c, nrhs);
  const size_t bi = (size_t)nrhs * c->L[level + 1].n() * 16, bo = (size_t)nrhs * c->L[level].n() * 16;
  const double2* i = in_dev(c, coarse, bi, where, 0);
  double2* o = out_dev(c, fine, bo, where, 1);
  if (prec == WCMG_F64) transfer_ext<double>(c, level, i, o, nrhs, false);
  else if (prec == WCMG_F32) transfer_ext<float>(c, level, i, o, nrhs, false);
  else throw Error(WCMG_ERR_ARG, "prec must be F64 or F32");
  out_finish(c, fine, o, bo, where);
  API_END(c)
}

extern "C++" {
template <typename R>
static void coarse_ext(wcmg_ctx* c, int level, const double2* in, double2* out, int nrhs) {
  Level& L = c->L[level];
  cplx<R>* a = ws<R>(L, "io_a", nrhs);
  cplx<R>* b = ws<R>(L, "io_b", nrhs);
  pack_level<R>(c, level, a, in, nrhs);
  apply_op<R>(c, level, b, a, nrhs);
  unpack_level<R>(c, level, out, b, nrhs);
}
}  // extern "C++"

int wcmg_apply_coarse(wcmg_ctx* c, int level, const void* in, void* out, int nrhs, int prec, int where,
                      void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 1, c->p.n_levels - 1);
  check_rhs(c, nrhs);
  const size_t bytes = (size_t)nrhs * c->L[level].n() * 16;
  const double2* i = in_dev(c, in, bytes, where, 0);
  double2* o = out_dev(c, out, bytes, where, 1);
  if (prec == WCMG_F64) coarse_ext<double>(c, level, i, o, nrhs);
  else if (prec == WCMG_F32) coarse_ext<float>(c, level, i, o, nrhs);
  else throw Error(WCMG_ERR_ARG, "prec must be F64 or F32");
  out_finish(c, out, o, bytes, where);
  API_END(c)
}

extern "C++" {
static void setup_from(wcmg_ctx* c, const double2* iv, wcmg_stats* st);
}

int wcmg_setup(wcmg_ctx* c, const void* init_vecs, int where, void* stream, wcmg_stats* st) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  if (!init_vecs) throw Error(WCMG_ERR_ARG, "init_vecs is required");
  size_t tot = 0;
  for (int l = 0; l + 1 < c->p.n_levels; ++l) tot += (size_t)c->L[l].nvec * c->L[l].n() * 16;
  setup_from(c, in_dev(c, init_vecs, tot, where, 2), st);
  API_END(c)
}

int wcmg_setup_seeded(wcmg_ctx* c, unsigned long long seed, void* stream, wcmg_stats* st) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_gauge) throw Error(WCMG_ERR_STATE, "gauge field not set");
  size_t tot = 0;
  for (int l = 0; l + 1 < c->p.n_levels; ++l) tot += (size_t)c->L[l].nvec * c->L[l].n() * 16;
  double2* iv = (double2*)c->stage[2].ensure(tot);
  long long off = 0;
  for (int l = 0; l + 1 < c->p.n_levels; ++l) {
    const long long n = c->L[l].n();
    launch_counter_gaussian(iv + off, n, c->L[l].nvec, seed, 1ULL + 1000ULL * l, c->st);
    off += (long long)c->L[l].nvec * n;
  }
  setup_from(c, iv, st);
  API_END(c)
}

extern "C++" {
static void setup_from(wcmg_ctx* c, const double2* iv, wcmg_stats* st) {
  if (st) std::memset(st, 0, sizeof(*st));
  c->prof.flush();
  wcmg_kstat k0[WCMG_NKCLASS];
  std::memcpy(k0, c->prof.k, sizeof(k0));
  c->coarse_its = 0;
  const long long l0 = launch_counter();
  if (inner64(c)) setup_all<double>(c, iv, st);
  else setup_all<float>(c, iv, st);
  check_device_waits(c);
  c->prof.flush();
  if (st) {
    kstat_delta(st->k, c->prof.k, k0);
    st->coarse_iterations = c->coarse_its;
    st->kernel_launches = launch_counter() - l0;
  }
}
}  // extern "C++"

int wcmg_mg_cycle(wcmg_ctx* c, const void* r, void* e, int nrhs, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_rhs(c, nrhs);
  const size_t bytes = (size_t)nrhs * c->L[0].n() * 16;
  const double2* i = in_dev(c, r, bytes, where, 0);
  double2* o = out_dev(c, e, bytes, where, 1);
  Level& L = c->L[0];
  if (inner64(c)) {
    double2* a = ws<double>(L, "io_a", nrhs);
    double2* b = ws<double>(L, "io_b", nrhs);
    pack_level<double>(c, 0, a, i, nrhs);
    cycle<double>(c, 0, b, a, nrhs);
    unpack_level<double>(c, 0, o, b, nrhs);
  } else {
    float2* a = ws<float>(L, "io_a", nrhs);
    float2* b = ws<float>(L, "io_b", nrhs);
    pack_level<float>(c, 0, a, i, nrhs);
    cycle<float>(c, 0, b, a, nrhs);
    unpack_level<float>(c, 0, o, b, nrhs);
  }
  out_finish(c, e, o, bytes, where);
  API_END(c)
}

extern "C++" {
template <typename R>
static int krylov_ext(wcmg_ctx* c, int level, int kind, const double2* b, double2* x, int nrhs, int sr, double tol,
                      int maxiter) {
  Level& L = c->L[level];
  cplx<R>* a = ws<R>(L, "io_a", nrhs);
  cplx<R>* y = ws<R>(L, "io_b", nrhs);
  pack_level<R>(c, level, a, b, nrhs);
  int its = 0;
  if (kind == 0) {
    mr<R>(c, level, y, a, nrhs, sr);
    its = sr;
  } else if (kind == 2) {
    sap<R>(c, level, y, a, nrhs, sr, c->p.sap_cycles);
    its = sr;
  } else {
    KrylovOut k = fgmres<R>(c, level, y, a, nrhs, sr, tol, maxiter, true, false, false);
    its = k.iterations;
  }
  unpack_level<R>(c, level, x, y, nrhs);
  return its;
}
}  // extern "C++"

int wcmg_krylov(wcmg_ctx* c, int level, int kind, const void* b, void* x, int nrhs, int steps_or_restart, double tol,
                int maxiter, int where, void* stream, int* iters_out) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 0, c->p.n_levels - 1);
  check_rhs(c, nrhs);
  if (kind != 0 && kind != 1 && kind != 2) throw Error(WCMG_ERR_ARG, "kind must be 0 (MR), 1 (GMRES) or 2 (SAP)");
  if (kind == 2 && level >= c->p.n_levels - 1) throw Error(WCMG_ERR_ARG, "SAP needs a level with aggregates");
  if (steps_or_restart < 1 || steps_or_restart > 64) throw Error(WCMG_ERR_ARG, "steps/restart out of range");
  const size_t bytes = (size_t)nrhs * c->L[level].n() * 16;
  const double2* i = in_dev(c, b, bytes, where, 0);
  double2* o = out_dev(c, x, bytes, where, 1);
  int its = inner64(c) ? krylov_ext<double>(c, level, kind, i, o, nrhs, steps_or_restart, tol, maxiter)
                       : krylov_ext<float>(c, level, kind, i, o, nrhs, steps_or_restart, tol, maxiter);
  out_finish(c, x, o, bytes, where);
  if (iters_out) *iters_out = its;
  API_END(c)
}

int wcmg_solve(wcmg_ctx* c, const void* b, void* x, int nrhs, int where, void* stream, wcmg_stats* st) {
  wcmg_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  o.zero_guess = 1;
  return wcmg_solve_ex(c, b, x, nrhs, &o, where, stream, st);
}

int wcmg_solve_ex(wcmg_ctx* c, const void* b, void* x, int nrhs, const wcmg_solve_opts* opts, int where,
                  void* stream, wcmg_stats* st) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_rhs(c, nrhs);
  if (!opts || (opts->zero_guess != 0 && opts->zero_guess != 1))
    throw Error(WCMG_ERR_ARG, "opts must be given with zero_guess 0 or 1");
  const bool guess = opts->zero_guess == 0;
  for (int l = 0; l + 1 < c->p.n_levels; ++l)
    if (!c->L[l].have_P || !c->L[l + 1].have_op) throw Error(WCMG_ERR_STATE, "setup not done");
  wcmg_stats local;
  if (!st) st = &local;
  const double ms_i = st->ms_setup_init, ms_r = st->ms_setup_refine;
  std::memset(st, 0, sizeof(*st));
  st->ms_setup_init = ms_i;
  st->ms_setup_refine = ms_r;
  c->prof.flush();
  wcmg_kstat k0[WCMG_NKCLASS];
  std::memcpy(k0, c->prof.k, sizeof(k0));
  c->coarse_its = 0;
  long long l0 = launch_counter();
  auto t0 = std::chrono::steady_clock::now();
  if (c->coarse_mode != WCMG_COARSE_MG) {
    if (!c->have_ptc) throw Error(WCMG_ERR_STATE, "learned coarse mode needs PTC weights");
    if (inner64(c)) throw Error(WCMG_ERR_ARG, "learned coarse modes need inner_prec F32");
  }
  c->learned_on = c->coarse_mode != WCMG_COARSE_MG;
  c->learned_fallback = false;
  c->learned_cycles = 0;
  Level& L = c->L[0];
  const size_t bytes = (size_t)nrhs * L.n() * 16;
  const double2* bi = in_dev(c, b, bytes, where, 0);
  double2* xo = out_dev(c, x, bytes, where, 1);
  double2* b64 = ws<double>(L, "sv_b", nrhs);
  double2* x64 = ws<double>(L, "sv_x", nrhs);
  pack_level<double>(c, 0, b64, bi, nrhs);
  if (guess) {  // x holds the initial guess on entry
    const double2* xi = static_cast<const double2*>(x);
    if (where == WCMG_HOST) {
      WCMG_CUDA(cudaMemcpyAsync(xo, x, bytes, cudaMemcpyHostToDevice, c->st));
      xi = xo;
    }
    pack_level<double>(c, 0, x64, xi, nrhs);
  }
  c->guess = guess;
  const bool want_graph = c->p.use_graphs && c->coarse_mode == WCMG_COARSE_MG;
  long long graph_kernels = 0;
  if (want_graph) graph_prepare(c, nrhs);
  if (want_graph && is_warm(c, nrhs)) {
    auto& G = c->graph;
    if (!G.exec || G.nrhs != nrhs || G.gen != graph_epoch() || G.guess != guess) {
      wcmg_ctx* cs[1] = {c};
      double2* xs[1] = {x64};
      const double2* bs[1] = {b64};
      const int nr[1] = {nrhs};
      const long long lc = launch_counter();
      capture_group(cs, 1, xs, bs, nr, G);
      G.nrhs = nrhs;
      G.guess = guess;
      l0 += launch_counter() - lc;  // captured, not launched
    }
    WCMG_CUDA(cudaGraphLaunch(G.exec, c->st));
    graph_stats(c, st);
    graph_kernels = st->kernel_launches;
  } else {
    if (inner64(c)) solve_f64(c, x64, b64, nrhs, st);
    else solve_mixed(c, x64, b64, nrhs, st);
    st->coarse_iterations = c->coarse_its;
    if (want_graph) c->warm_rhs.push_back(nrhs);
  }
  check_device_waits(c);
  st->true_residual = true_residual(c, x64, b64, nrhs);
  st->converged = st->true_residual <= c->p.outer_tol;
  unpack_level<double>(c, 0, xo, x64, nrhs);
  out_finish(c, x, xo, bytes, where);
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  auto t1 = std::chrono::steady_clock::now();
  st->ms_solve = std::chrono::duration<double, std::milli>(t1 - t0).count();
  c->prof.flush();
  kstat_delta(st->k, c->prof.k, k0);
  st->kernel_launches = graph_kernels + (launch_counter() - l0);
  st->learned_cycles = c->learned_cycles;
  st->learned_fallback = c->learned_fallback ? 1 : 0;
  c->learned_on = false;
  if (!st->converged) {
    c->err = "outer solver reached outer_maxiter";
    return WCMG_ERR_NOT_CONVERGED;
  }
  API_END(c)
}

int wcmg_solve_batch(wcmg_ctx* const* ctxs, int n, const void* const* b, void* const* x, const int* nrhs,
                     int where, void* stream, wcmg_stats* st) {
  if (!ctxs || n < 1 || !ctxs[0]) return WCMG_ERR_ARG;
  wcmg_ctx* c0 = ctxs[0];
  API_BEGIN(c0)
  if (!b || !x || !nrhs) throw Error(WCMG_ERR_ARG, "null argument");
  for (int i = 0; i < n; ++i) {
    wcmg_ctx* c = ctxs[i];
    if (!c) throw Error(WCMG_ERR_ARG, "null context");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == c) throw Error(WCMG_ERR_ARG, "context repeated in a batch");
    c->st = (cudaStream_t)stream;
    check_rhs(c, nrhs[i]);
    for (int l = 0; l + 1 < c->p.n_levels; ++l)
      if (!c->L[l].have_P || !c->L[l + 1].have_op) throw Error(WCMG_ERR_STATE, "setup not done");
    if (c->coarse_mode != WCMG_COARSE_MG) throw Error(WCMG_ERR_ARG, "batched solve needs the plain multigrid mode");
  }
  std::vector<wcmg_stats> local(n);
  auto S = [&](int i) -> wcmg_stats& { return st ? st[i] : local[i]; };
  long long l0 = launch_counter();
  auto t0 = std::chrono::steady_clock::now();
  std::vector<double2*> xs(n), xo(n);
  std::vector<const double2*> bs(n);
  std::vector<size_t> bytes(n);
  for (int i = 0; i < n; ++i) {
    wcmg_ctx* c = ctxs[i];
    const double mi = S(i).ms_setup_init, mr = S(i).ms_setup_refine;
    std::memset(&S(i), 0, sizeof(wcmg_stats));
    S(i).ms_setup_init = mi;
    S(i).ms_setup_refine = mr;
    c->coarse_its = 0;
    c->learned_on = false;
    c->guess = false;
    Level& L = c->L[0];
    bytes[i] = (size_t)nrhs[i] * L.n() * 16;
    const double2* bi = in_dev(c, b[i], bytes[i], where, 0);
    xo[i] = out_dev(c, x[i], bytes[i], where, 1);
    double2* b64 = ws<double>(L, "sv_b", nrhs[i]);
    xs[i] = ws<double>(L, "sv_x", nrhs[i]);
    bs[i] = b64;
    pack_level<double>(c, 0, b64, bi, nrhs[i]);
    graph_prepare(c, nrhs[i]);
  }
  bool warm = true;
  for (int i = 0; i < n; ++i) warm &= is_warm(ctxs[i], nrhs[i]);
  std::vector<long long> gk(n, 0);
  if (!warm) {
    for (int i = 0; i < n; ++i) {
      wcmg_ctx* c = ctxs[i];
      if (inner64(c)) solve_f64(c, xs[i], bs[i], nrhs[i], &S(i));
      else solve_mixed(c, xs[i], bs[i], nrhs[i], &S(i));
      S(i).coarse_iterations = c->coarse_its;
      if (!is_warm(c, nrhs[i])) c->warm_rhs.push_back(nrhs[i]);
    }
  } else {
    std::vector<const void*> key;
    for (int i = 0; i < n; ++i) {
      key.push_back(ctxs[i]);
      key.push_back(reinterpret_cast<const void*>((intptr_t)nrhs[i]));
    }
    auto& G = c0->batch;
    if (!G.exec || key != c0->batch_key || G.gen != graph_epoch()) {
      const long long lc = launch_counter();
      capture_group(const_cast<wcmg_ctx**>(ctxs), n, xs.data(), bs.data(), nrhs, G);
      c0->batch_key = key;
      l0 += launch_counter() - lc;
    }
    WCMG_CUDA(cudaGraphLaunch(G.exec, (cudaStream_t)stream));
    for (int i = 0; i < n; ++i) {
      graph_stats(ctxs[i], &S(i));
      gk[i] = S(i).kernel_launches;
    }
  }
  const long long eager = launch_counter() - l0;  // all contexts' host-launched kernels
  int rc = WCMG_OK;
  for (int i = 0; i < n; ++i) {
    wcmg_ctx* c = ctxs[i];
    check_device_waits(c);
    S(i).true_residual = true_residual(c, xs[i], bs[i], nrhs[i]);
    S(i).converged = S(i).true_residual <= c->p.outer_tol;
    unpack_level<double>(c, 0, xo[i], xs[i], nrhs[i]);
    out_finish(c, x[i], xo[i], bytes[i], where);
    if (!S(i).converged && rc == WCMG_OK) {
      rc = WCMG_ERR_NOT_CONVERGED;
      c0->err = "a context of the batch reached outer_maxiter";
    }
  }
  WCMG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  auto t1 = std::chrono::steady_clock::now();
  const double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  for (int i = 0; i < n; ++i) {
    S(i).ms_solve = ms;
    S(i).kernel_launches = gk[i] + (i == 0 ? eager : 0);
  }
  if (rc != WCMG_OK) return rc;
  API_END(c0)
}

// ---- coarse-apply tiles ----
extern "C++" {
// link storage kind of the full coarse apply of level l at `prec` (0 FP64, 1 FP32, 2 BF16, 3 FP16)
static int link_kind_for(wcmg_ctx* c, int l, int prec) {
  Level& L = c->L[l];
  if (!L.have_op) throw Error(WCMG_ERR_STATE, "coarse operator of level not built");
  if (prec == WCMG_F64) {
    if (!L.op64) throw Error(WCMG_ERR_ARG, "FP64 coarse apply needs FP64 links");
    return 0;
  }
  if (prec != WCMG_F32) throw Error(WCMG_ERR_ARG, "prec must be F64 or F32");
  const int lp = c->p.coarse_link_prec;
  if (L.low_valid && lp == WCMG_BF16) return 2;
  if (L.low_valid && lp == WCMG_F16) return 3;
  return 1;
}
static void tile_out(const Level::TileInfo& ti, wcmg_tile* o) {
  std::memset(o, 0, sizeof(*o));
  o->kind = ti.t.kind;
  o->rhs_per_cta = ti.t.rr;
  o->parts = ti.t.parts;
  o->threads = ti.t.threads;
  o->ntile = ti.t.ntile;
  o->stages = ti.t.stages;
  o->source = ti.source;
  o->candidates = ti.candidates;
  o->us = ti.us;
  o->us_default = ti.us_default;
}
}  // extern "C++"

int wcmg_get_coarse_tile(wcmg_ctx* c, int level, int nrhs, int prec, wcmg_tile* out) {
  API_BEGIN(c)
  check_level(c, level, 1, c->p.n_levels - 1);
  check_rhs(c, nrhs);
  if (!out) throw Error(WCMG_ERR_ARG, "out");
  Level& L = c->L[level];
  const int lk = link_kind_for(c, level, prec);
  auto it = L.tiles.find({nrhs, lk});
  Level::TileInfo ti;
  if (it != L.tiles.end()) ti = it->second;
  else ti.t = coarse_default_tile(L.nc, nrhs, ST_FULL, L.g.V, lk);
  tile_out(ti, out);
  API_END(c)
}

int wcmg_tune_coarse(wcmg_ctx* c, int level, int nrhs, int prec, int cold, void* stream, wcmg_tile* out) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_level(c, level, 1, c->p.n_levels - 1);
  check_rhs(c, nrhs);
  if (cold != 0 && cold != 1) throw Error(WCMG_ERR_ARG, "cold must be 0 or 1");
  Level& L = c->L[level];
  const int lk = link_kind_for(c, level, prec);
  Level::TileInfo ti;
  if (lk == 0) ti = tune_coarse<double, double2>(c, level, L.L64.p, nrhs, 0, cold);
  else if (lk == 2) ti = tune_coarse<float, bf16c>(c, level, L.Lbf.p, nrhs, 2, cold);
  else if (lk == 3) ti = tune_coarse<float, f16c>(c, level, L.Lh.p, nrhs, 3, cold);
  else {
    if (!L.L32_valid) {
      const long long n = (long long)L.g.V * L.nc * links_ld(L.nc);
      L.L32.ensure(n);
      launch_convert_links<double2, float2>(L.L32.p, L.L64.p, n, c->st);
      L.L32_valid = true;
      if (c->p.coarse_sigma3 && L.sigma3) build_links5_of<float2>(c, level, L.L32.p);
    }
    ti = tune_coarse<float, float2>(c, level, L.L32.p, nrhs, 1, cold);
  }
  L.tiles[{nrhs, lk}] = ti;
  ++graph_epoch();
  check_device_waits(c);
  if (out) tile_out(ti, out);
  API_END(c)
}

int wcmg_set_coarse_tile(wcmg_ctx* c, int level, int nrhs, int prec, const wcmg_tile* t) {
  API_BEGIN(c)
  check_level(c, level, 1, c->p.n_levels - 1);
  check_rhs(c, nrhs);
  if (!t) throw Error(WCMG_ERR_ARG, "tile");
  Level& L = c->L[level];
  const int lk = link_kind_for(c, level, prec);
  if (t->kind < 0) {
    L.tiles.erase({nrhs, lk});
  } else {
    Level::TileInfo ti;
    ti.t.kind = t->kind;
    ti.t.rr = t->rhs_per_cta;
    ti.t.parts = t->parts;
    ti.t.threads = t->threads;
    ti.t.ntile = t->ntile;
    ti.t.stages = t->stages;
    if (!coarse_tile_valid(ti.t, L.nc, nrhs, ST_FULL, lk)) throw Error(WCMG_ERR_ARG, "tile not valid for this level");
    if (ti.t.kind == 5 && !(c->p.coarse_sigma3 && L.sigma3 && L.l5_valid[lk]))
      throw Error(WCMG_ERR_ARG, "kind 5 needs params.coarse_sigma3 and a coarse operator built by the setup");
    ti.source = 2;
    L.tiles[{nrhs, lk}] = ti;
  }
  ++graph_epoch();
  API_END(c)
}

int wcmg_check_bounded_wait(wcmg_ctx* c, long long polls, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (polls < 0 || polls > (1LL << 26)) throw Error(WCMG_ERR_ARG, "polls must be 0 .. 2^26");
  c->tma_err.ensure(1);
  launch_wait_selftest(c->tma_err.p, polls, c->st);
  check_device_waits(c);
  throw Error(WCMG_ERR_STATE, "the self-test wait did not give up");
  API_END(c)
}

int wcmg_set_profile(wcmg_ctx* c, int mask) {
  API_BEGIN(c)
  c->prof.flush();
  c->p.profile = mask;
  c->prof.mask = mask;
  API_END(c)
}

int wcmg_get_opcounts(wcmg_ctx* c, long long* out) {
  API_BEGIN(c)
  if (!out) throw Error(WCMG_ERR_ARG, "null output");
  for (int k = 0; k < WCMG_NOPC; ++k)
    for (int l = 0; l < WCMG_MAX_LEVELS; ++l) out[k * WCMG_MAX_LEVELS + l] = c->opc[k][l];
  API_END(c)
}

int wcmg_get_kstats(wcmg_ctx* c, wcmg_kstat* out) {
  API_BEGIN(c)
  if (!out) throw Error(WCMG_ERR_ARG, "out");
  c->prof.flush();
  std::memcpy(out, c->prof.k, sizeof(c->prof.k));
  API_END(c)
}

int wcmg_ptc_set_weights(wcmg_ctx* c, const void* W, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  const double2* w = in_dev(c, W, sizeof(double2) * WCMG_PTC_NWEIGHTS, where, 0);
  ptc_alloc(c);
  launch_convert<double, float>(c->ptcW.p, w, WCMG_PTC_NWEIGHTS, c->st);
  c->have_ptc = true;
  WCMG_CUDA(cudaStreamSynchronize(c->st));
  API_END(c)
}

int wcmg_ptc_get_weights(wcmg_ctx* c, void* W, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!c->have_ptc) throw Error(WCMG_ERR_STATE, "PTC weights not set");
  const size_t bytes = sizeof(double2) * WCMG_PTC_NWEIGHTS;
  double2* o = out_dev(c, W, bytes, where, 1);
  launch_convert<float, double>(o, c->ptcW.p, WCMG_PTC_NWEIGHTS, c->st);
  out_finish(c, W, o, bytes, where);
  API_END(c)
}

int wcmg_ptc_forward(wcmg_ctx* c, const void* in, void* out, int nrhs, int where, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_rhs(c, nrhs);
  Level& L = c->L[0];
  const size_t bytes = (size_t)nrhs * L.n() * 16;
  const double2* i = in_dev(c, in, bytes, where, 0);
  double2* o = out_dev(c, out, bytes, where, 1);
  float2* a = ws<float>(L, "io_a", nrhs);
  float2* b = ws<float>(L, "io_b", nrhs);
  pack_level<float>(c, 0, a, i, nrhs);
  ptc_forward(c, b, a, nrhs);
  unpack_level<float>(c, 0, o, b, nrhs);
  out_finish(c, out, o, bytes, where);
  API_END(c)
}

int wcmg_ptc_backward(wcmg_ctx* c, const void* in, const void* gout, void* gin, void* gW, int nrhs, int where,
                      void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  check_rhs(c, nrhs);
  if (!c->have_ptc) throw Error(WCMG_ERR_STATE, "PTC weights not set");
  Level& L = c->L[0];
  const size_t bytes = (size_t)nrhs * L.n() * 16, wbytes = sizeof(double2) * WCMG_PTC_NWEIGHTS;
  const double2* i = in_dev(c, in, bytes, where, 0);
  const double2* g = in_dev(c, gout, bytes, where, 1);
  float2* a = ws<float>(L, "io_a", nrhs);
  float2* b = ws<float>(L, "io_b", nrhs);
  float2* d = ws<float>(L, "io_c", nrhs);
  pack_level<float>(c, 0, a, i, nrhs);
  pack_level<float>(c, 0, b, g, nrhs);
  ptc_backward(c, a, b, d, nrhs);
  double2* go = out_dev(c, gin, bytes, where, 2);
  unpack_level<float>(c, 0, go, d, nrhs);
  out_finish(c, gin, go, bytes, where);
  double2* wo = (where == WCMG_DEVICE) ? (double2*)gW : (double2*)c->stage[1].ensure(wbytes);
  launch_convert<float, double>(wo, c->ptcG.p, WCMG_PTC_NWEIGHTS, c->st);
  out_finish(c, gW, wo, wbytes, where);
  API_END(c)
}

int wcmg_ptc_train(wcmg_ctx* c, const wcmg_train_opts* opts, wcmg_train_stats* st, void* stream) {
  API_BEGIN(c)
  c->st = (cudaStream_t)stream;
  if (!opts || !st) throw Error(WCMG_ERR_ARG, "opts and st are required");
  std::memset(st, 0, sizeof(*st));
  ptc_train(c, opts, st);
  check_device_waits(c);
  c->prof.flush();
  API_END(c)
}

int wcmg_set_coarse_mode(wcmg_ctx* c, int mode, double fallback_ratio) {
  API_BEGIN(c)
  if (mode < WCMG_COARSE_MG || mode > WCMG_COARSE_LEARNED) throw Error(WCMG_ERR_ARG, "coarse mode");
  c->coarse_mode = mode;
  c->fallback_ratio = fallback_ratio;
  API_END(c)
}

int wcmg_save_net(wcmg_ctx* c, const char* path) {
  API_BEGIN(c)
  if (!path) throw Error(WCMG_ERR_ARG, "path");
  if (!c->have_ptc) throw Error(WCMG_ERR_STATE, "no PTC weights to save");
  std::vector<float2> h(WCMG_PTC_NWEIGHTS);
  WCMG_CUDA(cudaDeviceSynchronize());
  WCMG_CUDA(cudaMemcpy(h.data(), c->ptcW.p, sizeof(float2) * h.size(), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) throw Error(WCMG_ERR_ARG, std::string("cannot open ") + path);
  const char magic[8] = {'W', 'C', 'M', 'G', 'N', 'E', 'T', '1'};
  const int hdr[4] = {WCMG_PTC_HIDDEN, WCMG_PTC_NWEIGHTS, 4 /* bytes per real */, 0};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 4, f) == 4 &&
            std::fwrite(h.data(), sizeof(float2), h.size(), f) == h.size();
  ok &= std::fclose(f) == 0;
  if (!ok) throw Error(WCMG_ERR_ARG, std::string("cannot write ") + path);
  API_END(c)
}

int wcmg_load_net(wcmg_ctx* c, const char* path) {
  API_BEGIN(c)
  if (!path) throw Error(WCMG_ERR_ARG, "path");
  FILE* f = std::fopen(path, "rb");
  if (!f) throw Error(WCMG_ERR_ARG, std::string("cannot open ") + path);
  char magic[8] = {};
  int hdr[4] = {};
  std::vector<float2> h(WCMG_PTC_NWEIGHTS);
  const bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "WCMGNET1", 8) == 0 &&
                  std::fread(hdr, sizeof(int), 4, f) == 4 && hdr[0] == WCMG_PTC_HIDDEN &&
                  hdr[1] == WCMG_PTC_NWEIGHTS && hdr[2] == 4 &&
                  std::fread(h.data(), sizeof(float2), h.size(), f) == h.size();
  std::fclose(f);
  if (!ok) throw Error(WCMG_ERR_ARG, std::string("not a PTC network file of this shape: ") + path);
  ptc_alloc(c);
  WCMG_CUDA(cudaDeviceSynchronize());
  WCMG_CUDA(cudaMemcpy(c->ptcW.p, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice));
  c->have_ptc = true;
  API_END(c)
}

int wcmg_save_setup(wcmg_ctx* c, const char* path) {
  API_BEGIN(c)
  if (!path) throw Error(WCMG_ERR_ARG, "path");
  FILE* f = std::fopen(path, "wb");
  if (!f) throw Error(WCMG_ERR_ARG, std::string("cannot open ") + path);
  const char magic[8] = {'W', 'C', 'M', 'G', 'S', 'E', 'T', '1'};
  std::fwrite(magic, 1, 8, f);
  std::fwrite(&c->p.n_levels, sizeof(int), 1, f);
  std::fwrite(c->p.dims, sizeof(int), 4, f);
  std::fwrite(c->p.nvec, sizeof(int), WCMG_MAX_LEVELS - 1, f);
  std::vector<double2> h;
  for (int l = 0; l + 1 < c->p.n_levels; ++l) {
    Level& L = c->L[l];
    if (!L.have_P || !c->L[l + 1].have_op) { std::fclose(f); throw Error(WCMG_ERR_STATE, "setup not done"); }
    const size_t nv = (size_t)L.nvec * L.n();
    h.resize(nv);
    double2* d = ws<double>(L, "io_a", L.nvec);
    if (L.fine) launch_unpack_fine<double>(d, L.v64.p, L.g.d_perm.p, L.g.V, L.nvec, c->st);
    else launch_unpack_coarse<double>(d, L.v64.p, L.g.d_perm.p, L.g.V, L.nc, L.nvec, c->st);
    WCMG_CUDA(cudaMemcpyAsync(h.data(), d, nv * 16, cudaMemcpyDeviceToHost, c->st));
    WCMG_CUDA(cudaStreamSynchronize(c->st));
    std::fwrite(h.data(), 16, nv, f);
  }
  for (int l = 1; l < c->p.n_levels; ++l) {
    Level& L = c->L[l];
    const int nb = L.nc;
    const size_t na = (size_t)9 * L.g.V * nb * nb;
    h.resize(na);
    DevBuf<double2> tmp;
    tmp.ensure(na);
    if (L.op64) launch_unpack_links<double2>(tmp.p, L.L64.p, L.g.d_perm.p, L.g.V, nb, c->st);
    else launch_unpack_links<float2>(tmp.p, L.L32.p, L.g.d_perm.p, L.g.V, nb, c->st);
    WCMG_CUDA(cudaMemcpyAsync(h.data(), tmp.p, na * 16, cudaMemcpyDeviceToHost, c->st));
    WCMG_CUDA(cudaStreamSynchronize(c->st));
    std::fwrite(h.data(), 16, na, f);
  }
  std::fclose(f);
  API_END(c)
}

int wcmg_load_setup(wcmg_ctx* c, const char* path) {
  API_BEGIN(c)
  if (!path) throw Error(WCMG_ERR_ARG, "path");
  FILE* f = std::fopen(path, "rb");
  if (!f) throw Error(WCMG_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int nl, dims[4], nvec[WCMG_MAX_LEVELS - 1];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "WCMGSET1", 8) == 0 &&
            std::fread(&nl, sizeof(int), 1, f) == 1 && std::fread(dims, sizeof(int), 4, f) == 4 &&
            std::fread(nvec, sizeof(int), WCMG_MAX_LEVELS - 1, f) == WCMG_MAX_LEVELS - 1;
  ok = ok && nl == c->p.n_levels && std::memcmp(dims, c->p.dims, sizeof(dims)) == 0;
  for (int l = 0; ok && l + 1 < nl; ++l) ok = nvec[l] == c->p.nvec[l];
  if (!ok) { std::fclose(f); throw Error(WCMG_ERR_ARG, "setup file does not match the context"); }
  std::vector<double2> h;
  for (int l = 0; l + 1 < nl; ++l) {
    Level& L = c->L[l];
    const size_t nv = (size_t)L.nvec * L.n();
    h.resize(nv);
    if (std::fread(h.data(), 16, nv, f) != nv) { std::fclose(f); throw Error(WCMG_ERR_ARG, "truncated setup file"); }
    double2* d = ws<double>(L, "io_a", L.nvec);
    WCMG_CUDA(cudaMemcpyAsync(d, h.data(), nv * 16, cudaMemcpyHostToDevice, c->st));
    L.v64.ensure(nv);
    if (L.fine) launch_pack_fine<double>(L.v64.p, d, L.g.d_perm.p, L.g.V, L.nvec, c->st);
    else launch_pack_coarse<double>(L.v64.p, d, L.g.d_perm.p, L.g.V, L.nc, L.nvec, c->st);
    L.raw64.ensure(nv);
    copy_fields<double>(c, L.raw64.p, L.v64.p, (long long)nv);
    if (!inner64(c)) {
      L.raw32.ensure(nv);
      launch_convert<double, float>(L.raw32.p, L.v64.p, (long long)nv, c->st);
    }
    L.v32_valid = false;
    L.have_P = true;
    WCMG_CUDA(cudaStreamSynchronize(c->st));
  }
  for (int l = 1; l < nl; ++l) {
    Level& L = c->L[l];
    const int nb = L.nc;
    const size_t na = (size_t)9 * L.g.V * nb * nb;
    h.resize(na);
    if (std::fread(h.data(), 16, na, f) != na) { std::fclose(f); throw Error(WCMG_ERR_ARG, "truncated setup file"); }
    int rc = wcmg_set_coarse_links(c, l, h.data(), WCMG_HOST, c->st);
    if (rc) { std::fclose(f); throw Error(rc, c->err); }
    if (!inner64(c)) {
      // links were produced in FP32: keep FP32 arithmetic on the FP32-rounded values
      L.op64 = false;
    }
  }
  std::fclose(f);
  API_END(c)
}

}  // extern "C"
