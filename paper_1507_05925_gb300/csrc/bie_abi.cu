// C ABI of libbie2d: context, workspace, argument staging and the solver
// drivers (restarted GMRES in FP64, and FP64 iterative refinement around
// GMRES with FP32 pair sums).  Every step of the path runs in the kernels of
// this library; the host only orders launches and reads the convergence state.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <initializer_list>
#include <map>
#include <mutex>
#include <atomic>
#include <string>
#include <vector>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"

using namespace bie;

namespace {
// weight alpha of the per-body completion used inside the FP32 inner solves
constexpr double kInnerCompletionWeight = 1.0;

// FMM schedules chosen by bie_tune_fmm, per device and shape (M, kind, order)
std::mutex g_fmm_mu;
std::map<std::array<int, 4>, bie::FmmSchedule> g_fmm_sched;
std::array<int, 4> fmm_key(int M, int kind, int order) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, M, kind, order};
}
}  // namespace

namespace bie {
FmmSchedule fmm_schedule(int M, int kind, int order) {
  std::lock_guard<std::mutex> lk(g_fmm_mu);
  auto it = g_fmm_sched.find(fmm_key(M, kind, order));
  if (it != g_fmm_sched.end()) return it->second;
  return FmmSchedule{kDefaultLeafNodes, std::max(2, (order + 1) / 2)};
}
}  // namespace bie

namespace bie {
static std::atomic<long long> g_launches{0};
// launches noted by this thread (a capture counts its own kernels while other
// server threads launch)
static thread_local long long t_launches = 0;
void note_launches(int k) {
  g_launches.fetch_add(k, std::memory_order_relaxed);
  t_launches += k;
}
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launches() { return t_launches; }
}  // namespace bie

struct bie_ctx {
  int device = 0;
  size_t cap = 0;
  char* ws = nullptr;
  size_t ws_size = 0;
  KState* h_state = nullptr;  // pinned mirror of the device solver state
  double* h_small = nullptr;  // pinned scratch for small read-backs
  std::string err;
  // pair-sum timing (bie_profile)
  struct Timing {
    cudaEvent_t a, b;
    int prec, kind;
    double pairs;
    bool valid;
  };
  bool prof = false;
  long long launch_mark = 0;
  bie_profile_counters counters{};
  std::vector<cudaEvent_t> pool;
  std::vector<Timing> pending;
  // CUDA graphs of one GMRES iteration, keyed by everything their kernels read
  struct IterGraph {
    long long key[12];
    cudaGraphExec_t exec;
    long long kernels;  // per iteration
    int last_cycle;     // iterations of the last cycle replayed from it (0: none yet)
  };
  std::vector<IterGraph> graphs;
  int graph_replay = 0;  // launch mode of the last GMRES cycle (bie_info.graph_replay)
  bie::FmmState* fmm = nullptr;  // quadtree of the last FMM call
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int fail(bie_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError(); /* a non-sticky error must not fail the next call */           \
      return fail(ctx, BIE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                    \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device memory of a device other than dev (managed memory is reachable from
// every device and passes).  Such an array is rejected before any kernel
// could dereference it: without peer access that would be an illegal address.
bool foreign_device_ptr(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice && at.device != dev;
}

int check_local(bie_ctx* ctx, std::initializer_list<const void*> ptrs, const char* what) {
  for (const void* p : ptrs)
    if (foreign_device_ptr(p, ctx->device))
      return fail(ctx, BIE_ERR_INVALID, std::string(what) + " is device memory of another device than the context's");
  return BIE_OK;
}

// Bump allocator over the context workspace: a sizing pass (base == nullptr)
// and a carving pass.
struct Arena {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Work {
  Geo g;
  int kind = 0, n = 0, m = 50;
  long long ld = 0;
  // raw input staging
  int* body_start = nullptr;
  double *x = nullptr, *y = nullptr, *dx = nullptr, *dy = nullptr, *ddx = nullptr, *ddy = nullptr;
  double *ipt = nullptr, *load = nullptr, *io_in = nullptr, *io_out = nullptr;
  // solver
  float* VF = nullptr;  // FP32 copy of the basis for the FP32 inner solves (single systems)
  double *V = nullptr, *f = nullptr, *xs = nullptr, *r = nullptr, *d = nullptr, *rin = nullptr, *ytmp = nullptr;
  double* rc = nullptr;
  // block-Jacobi preconditioner of the inner solves
  long long* bj_off = nullptr;
  int* bj_pairs = nullptr;
  bj_t* bj_blocks = nullptr;
  int* bj_fallbacks = nullptr;  // device counter of bodies left with the identity block
  double* zbuf = nullptr;
  double* arn = nullptr;  // per-CTA partials of the fused Arnoldi step
  // batched solves: per-body problem node range, first body and first entry of
  // each problem, and the problems' right-hand-side scales
  int2* prange = nullptr;
  int* pbody = nullptr;
  long long* pnode = nullptr;
  double* pscale = nullptr;
  double* pnorm = nullptr;  // per-problem residual norms of the refinement
  double* pnet = nullptr;   // per-problem net load and largest |load|
  SmallInfo* sinfo = nullptr;  // one-launch small-problem solves: per-problem counts
  // batched GMRES (one Krylov space per problem): element ranges of the fused
  // Arnoldi step and per-problem state; seg.P == 0 for a single system
  SegArgs seg;
  PState* ps = nullptr;
  long long* ibeg = nullptr;
  int *iprob = nullptr, *pitem = nullptr, *bprob = nullptr;
  int seg_grid = 1;
  long long max_plen = 0;
  int bj_max_nb = 0;
  double *partial = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *yv = nullptr;
  double *part = nullptr, *outpart = nullptr, *outv = nullptr, *cres = nullptr;
  KState* st = nullptr;
  PairPlan plan64, plan32, planff;
  int P = 1, grid = 1;
};

void carve(Arena& A, Work& w, int N, int M, int kind, int m, bool solve, bool stage_in, bool stage_ipt,
           bool stage_load, bool stage_io, long long bj_floats = 0, int nprob = 0, const int* bs = nullptr,
           const int* pb = nullptr) {
  const int comps = kind + 1;
  const long long n = (long long)M * comps;
  w.kind = kind;
  w.n = (int)n;
  w.m = m;
  w.ld = (n + 31) & ~31LL;
  Geo& g = w.g;
  g.N = N;
  g.M = M;
  w.body_start = A.take<int>(N + 1);
  g.body_of = A.take<int>(M);
  g.x = A.take<double>(M);
  g.y = A.take<double>(M);
  g.nx = A.take<double>(M);
  g.ny = A.take<double>(M);
  g.w = A.take<double>(M);
  g.sw = A.take<double>(M);
  g.kappa = A.take<double>(M);
  g.pf = A.take<float4>(M);
  g.nf = A.take<float2>(M);
  g.wkf = A.take<float2>(M);
  g.xff = A.take<float4>(M);
  g.xfl = A.take<float2>(M);
  g.nff = A.take<float4>(M);
  g.qf = A.take<float>(2 * (size_t)M);
  g.len = A.take<double>(N);
  g.xc = A.take<double>(N);
  g.yc = A.take<double>(N);
  g.W = A.take<double>(N);
  g.zx = A.take<double>(N);
  g.zy = A.take<double>(N);
  g.delta = A.take<double>(N);
  g.wind = A.take<double>(N);
  g.bbox = A.take<float4>(N);
  g.qscale = A.take<double>(2);
  if (stage_in) {
    w.x = A.take<double>(M);
    w.y = A.take<double>(M);
    w.dx = A.take<double>(M);
    w.dy = A.take<double>(M);
    w.ddx = A.take<double>(M);
    w.ddy = A.take<double>(M);
  }
  if (stage_ipt) w.ipt = A.take<double>(2 * N);
  if (stage_load) w.load = A.take<double>(3 * N);
  if (stage_io) {
    w.io_in = A.take<double>(n);
    w.io_out = A.take<double>(n);
  }
  if (nprob > 1) {
    w.plan64 = plan_pairs_batch(bs, N, pb, nprob, kind, 0);
    w.plan32 = plan_pairs_batch(bs, N, pb, nprob, kind, 1);
    w.planff = plan_pairs_batch(bs, N, pb, nprob, kind, 2);
  } else {
    w.plan64 = plan_pairs(M, kind, 0);
    w.plan32 = plan_pairs(M, kind, 1);
    w.planff = plan_pairs(M, kind, 2);
  }
  // problems solved as one system share every Krylov array; nseg copies of the
  // Hessenberg and rotation arrays with one Krylov space per problem
  const int nseg = nprob > 1 ? nprob : 1;
  long long arn_units = 0;
  if (nprob > 0) {  // a batch (of one or more problems)
    w.pbody = A.take<int>(nprob + 1);
    w.pnode = A.take<long long>(nprob + 1);
    w.pscale = A.take<double>(nprob);
    w.pnorm = A.take<double>(nprob);
    w.pnet = A.take<double>(2 * nprob);
    w.sinfo = A.take<SmallInfo>(nprob);
  }
  if (nprob > 1) {
    w.prange = A.take<int2>(N);
    const int items = kMaxVecGrid + nprob;  // ranges: at most grid + one per problem
    w.ps = A.take<PState>(nprob);
    w.ibeg = A.take<long long>(items + 1);
    w.iprob = A.take<int>(items);
    w.pitem = A.take<int>(nprob + 1);
    w.bprob = A.take<int>(N);
    arn_units = items;
  }
  const int S = std::max(std::max(w.plan64.S, w.plan32.S), w.planff.S);
  w.partial = A.take<double>((size_t)S * n);
  w.grid = vec_grid(n);
  w.part = A.take<double>((size_t)w.grid * 201 + 64);
  // per-CTA partials of the Arnoldi step: its grid is at most max(vec_grid, N + 1) CTAs
  const long long arn_grid = std::max<long long>(w.grid, std::min<long long>((long long)N + 1, kMaxVecGrid));
  w.arn = A.take<double>((size_t)3 * std::max<long long>(arn_grid, arn_units) * 201 + 64);
  w.st = A.take<KState>(1);
  if (solve) {
    w.V = A.take<double>((size_t)(m + 1) * w.ld);
    if (nprob <= 1) w.VF = A.take<float>((size_t)(m + 1) * w.ld);
    w.f = A.take<double>(n);
    w.xs = A.take<double>(n);
    w.r = A.take<double>(n);
    w.d = A.take<double>(n);
    w.rin = A.take<double>(n);
    w.ytmp = A.take<double>(n);
    w.rc = A.take<double>(n);
    w.H = A.take<double>((size_t)nseg * (m + 1) * m);
    w.cs = A.take<double>((size_t)nseg * m);
    w.sn = A.take<double>((size_t)nseg * m);
    w.gv = A.take<double>((size_t)nseg * (m + 1));
    w.yv = A.take<double>((size_t)nseg * (m + 1));
    w.P = output_splits(g, kind);
    const int targets = kind == 0 ? N : 3 * N;
    w.outpart = A.take<double>((size_t)w.P * targets * comps + N + 2);
    w.outv = A.take<double>(3 * N);
    w.cres = A.take<double>(1);
    if (bj_floats > 0) {
      w.bj_off = A.take<long long>(N + 1);
      w.bj_pairs = A.take<int>(N);
      w.bj_blocks = A.take<bj_t>((size_t)bj_floats);
      w.bj_fallbacks = A.take<int>(1);
      w.zbuf = A.take<double>(n);
    }
  }
}

// Stream-ordered (cudaMallocAsync) so that growing one context's workspace
// never synchronises the device under other contexts' work.
int ensure_ws(bie_ctx* ctx, size_t need, cudaStream_t s) {
  if (need <= ctx->ws_size) return BIE_OK;
  if (ctx->cap && need > ctx->cap)
    return fail(ctx, BIE_ERR_NOMEM, "workspace of " + std::to_string(need) + " bytes exceeds the cap of " +
                                        std::to_string(ctx->cap));
  if (ctx->ws) {
    cudaFreeAsync(ctx->ws, s);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
  }
  for (auto& gi : ctx->graphs) cudaGraphExecDestroy(gi.exec);  // their pointers are stale
  ctx->graphs.clear();
  CK(cudaMallocAsync(reinterpret_cast<void**>(&ctx->ws), need, s));
  ctx->ws_size = need;
  return BIE_OK;
}

// Copies a host array into staging (or passes a device pointer through).
template <class T>
int stage_in(bie_ctx* ctx, const T* src, T* staging, size_t count, const T** out, cudaStream_t s) {
  if (is_device_ptr(src)) {
    *out = src;
    return BIE_OK;
  }
  CK(cudaMemcpyAsync(staging, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = staging;
  return BIE_OK;
}

// Host-side argument checks; fills host copy of body_start.
int validate(bie_ctx* ctx, const bie_geometry* geom, std::vector<int>& bs) {
  if (!ctx) return BIE_ERR_INVALID;
  if (!geom) return fail(ctx, BIE_ERR_INVALID, "geometry is NULL");
  if (geom->n_bodies < 1) return fail(ctx, BIE_ERR_INVALID, "n_bodies must be >= 1");
  if (!geom->body_start || !geom->x || !geom->y || !geom->dx || !geom->dy || !geom->ddx || !geom->ddy)
    return fail(ctx, BIE_ERR_INVALID, "a geometry array is NULL");
  if (int rc = check_local(ctx, {geom->body_start, geom->x, geom->y, geom->dx, geom->dy, geom->ddx, geom->ddy,
                                 geom->interior_pt}, "a geometry array"))
    return rc;
  const int N = geom->n_bodies;
  bs.resize(N + 1);
  if (is_device_ptr(geom->body_start)) {
    CK(cudaMemcpy(bs.data(), geom->body_start, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  } else {
    memcpy(bs.data(), geom->body_start, (N + 1) * sizeof(int));
  }
  if (bs[0] != 0) return fail(ctx, BIE_ERR_INVALID, "body_start[0] must be 0");
  for (int i = 0; i < N; ++i)
    if (bs[i + 1] - bs[i] < 8)
      return fail(ctx, BIE_ERR_INVALID, "body " + std::to_string(i) + " has fewer than 8 nodes");
  if ((long long)bs[N] * 2 > 0x7fffffffLL) return fail(ctx, BIE_ERR_INVALID, "too many nodes");
  return BIE_OK;
}

// Stage the inputs and the geometry; check that the interior points lie inside.
int setup(bie_ctx* ctx, const bie_geometry* geom, const std::vector<int>& bs, Work& w, cudaStream_t s) {
  const int N = geom->n_bodies, M = bs[N];
  CK(cudaMemcpyAsync(w.body_start, bs.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  w.g.body_start = w.body_start;
  const double *x, *y, *dx, *dy, *ddx, *ddy, *ipt = nullptr;
  int rc;
  if ((rc = stage_in(ctx, geom->x, w.x, M, &x, s)) ||
      (rc = stage_in(ctx, geom->y, w.y, M, &y, s)) ||
      (rc = stage_in(ctx, geom->dx, w.dx, M, &dx, s)) ||
      (rc = stage_in(ctx, geom->dy, w.dy, M, &dy, s)) ||
      (rc = stage_in(ctx, geom->ddx, w.ddx, M, &ddx, s)) ||
      (rc = stage_in(ctx, geom->ddy, w.ddy, M, &ddy, s)))
    return rc;
  if (geom->interior_pt && (rc = stage_in(ctx, geom->interior_pt, w.ipt, 2 * (size_t)N, &ipt, s)))
    return rc;
  CK(stage_geometry(w.g, x, y, dx, dy, ddx, ddy, ipt, s));
  return BIE_OK;
}

// Batched solves: P independent problems of one kind, solved as one
// block-diagonal system.
struct BatchIn {
  int P;
  const bie_geometry* geoms;   // [P]
  const double* const* loads;  // [P]
  double* const* outs;         // [P]
  bie_info* infos;             // [P] or nullptr
  int* status;                 // [P] or nullptr
};

// Stage the problems one after another (host or device inputs) and the tables
// that keep every pair and output sum inside its own problem.
int batch_setup(bie_ctx* ctx, const BatchIn& b, const std::vector<int>& bs, const std::vector<int>& pb,
                bool ipt, Work& w, cudaStream_t s) {
  const int N = (int)bs.size() - 1, P = b.P, c = w.kind + 1;
  const long long M = bs[N];
  const int per = w.kind == 0 ? 1 : 3;  // load entries per body
  CK(cudaMemcpyAsync(w.body_start, bs.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  w.g.body_start = w.body_start;
  // geometry arrays, interior points and loads: device sources gathered by one
  // kernel, host sources packed and copied once per array (before the gather,
  // which then overwrites the device-sourced parts)
  double* dst[6] = {w.x, w.y, w.dx, w.dy, w.ddx, w.ddy};
  const long long ipt_off = 6 * M, load_off = 6 * M + 2LL * N;
  std::vector<double> pack;
  bool from_host[8] = {false, false, false, false, false, false, false, false};
  std::vector<CopySeg> segs;
  auto take = [&](int slot, const double* src, double* to, long long count, long long pack_at) {
    if (count <= 0) return;
    if (is_device_ptr(src)) {
      segs.push_back(CopySeg{src, to, 2 * count});
    } else {
      if (pack.empty()) pack.resize(load_off + (size_t)per * N);
      memcpy(pack.data() + pack_at, src, count * sizeof(double));
      from_host[slot] = true;
    }
  };
  for (int p = 0; p < P; ++p) {
    const bie_geometry& g = b.geoms[p];
    const long long off = bs[pb[p]], Mp = bs[pb[p + 1]] - bs[pb[p]], Np = pb[p + 1] - pb[p];
    const double* src[6] = {g.x, g.y, g.dx, g.dy, g.ddx, g.ddy};
    for (int k = 0; k < 6; ++k) take(k, src[k], dst[k] + off, Mp, k * M + off);
    if (ipt) take(6, g.interior_pt, w.ipt + 2 * pb[p], 2 * Np, ipt_off + 2 * pb[p]);
    take(7, b.loads[p], w.load + (long long)per * pb[p], per * Np, load_off + (long long)per * pb[p]);
  }
  for (int k = 0; k < 6; ++k)
    if (from_host[k]) CK(cudaMemcpyAsync(dst[k], pack.data() + k * M, M * sizeof(double), cudaMemcpyHostToDevice, s));
  if (from_host[6])
    CK(cudaMemcpyAsync(w.ipt, pack.data() + ipt_off, 2 * N * sizeof(double), cudaMemcpyHostToDevice, s));
  if (from_host[7])
    CK(cudaMemcpyAsync(w.load, pack.data() + load_off, (size_t)per * N * sizeof(double), cudaMemcpyHostToDevice,
                       s));
  CK(gather_segments(segs, s));
  std::vector<int2> pr(N);
  std::vector<long long> pn(P + 1);
  for (int p = 0; p < P; ++p) {
    for (int i = pb[p]; i < pb[p + 1]; ++i) pr[i] = make_int2(bs[pb[p]], bs[pb[p + 1]]);
    pn[p] = (long long)bs[pb[p]] * c;
  }
  pn[P] = (long long)bs[N] * c;
  // one problem needs no masking: its pair sums run as a single solve's
  if (P > 1) CK(cudaMemcpyAsync(w.prange, pr.data(), N * sizeof(int2), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.pbody, pb.data(), (P + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(w.pnode, pn.data(), (P + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
  w.g.prange = P > 1 ? w.prange : nullptr;
  w.g.pbody = w.pbody;
  w.g.nprob = P;
  w.g.pnet = w.pnet;
  w.g.pairs = 0.0;
  for (int p = 0; p < P; ++p) {
    const double mp = bs[pb[p + 1]] - bs[pb[p]];
    w.g.pairs += mp * (mp - 1.0);
  }
  std::vector<long long> ib;
  std::vector<int> ip, pi, bp;
  if (P > 1) {
    // element ranges of the batched Arnoldi step: about n / grid entries each
    // (at least 512), none crossing a problem
    w.seg_grid = arnoldi_seg_grid(pn[P]);
    const long long L = std::max<long long>(512, (pn[P] + w.seg_grid - 1) / w.seg_grid);
    pi.resize(P + 1);
    bp.resize(N);
    for (int p = 0; p < P; ++p) {
      pi[p] = (int)ip.size();
      const long long len = pn[p + 1] - pn[p];
      const long long k = std::max<long long>(1, (len + L - 1) / L);
      for (long long t = 0; t < k; ++t) {
        ib.push_back(pn[p] + len * t / k);
        ip.push_back(p);
      }
      for (int i = pb[p]; i < pb[p + 1]; ++i) bp[i] = p;
      w.max_plen = std::max(w.max_plen, len);
    }
    pi[P] = (int)ip.size();
    ib.push_back(pn[P]);
    if ((int)ip.size() > kMaxVecGrid + P) return fail(ctx, BIE_ERR_INVALID, "batch: internal range count");
    CK(cudaMemcpyAsync(w.ibeg, ib.data(), ib.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.iprob, ip.data(), ip.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.pitem, pi.data(), pi.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(w.bprob, bp.data(), bp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    w.seg.P = P;
    w.seg.nitem = (int)ip.size();
    w.seg.pnode = w.pnode;
    w.seg.ibeg = w.ibeg;
    w.seg.iprob = w.iprob;
    w.seg.pitem = w.pitem;
    w.seg.bprob = w.bprob;
    w.seg.ps = w.ps;
  }
  CK(stage_geometry(w.g, w.x, w.y, w.dx, w.dy, w.ddx, w.ddy, ipt ? w.ipt : nullptr, s));
  CK(cudaStreamSynchronize(s));  // the host tables above must outlive their copies
  return BIE_OK;
}

// Batched solves: every problem's argument checks, and the concatenated
// body_start (body offsets) and first body of each problem.  Device body_start
// arrays are gathered by one kernel and read back once.
int validate_batch(bie_ctx* ctx, const BatchIn& b, std::vector<int>& bs, std::vector<int>& pb, bool& has_ipt,
                   cudaStream_t s) {
  const int P = b.P;
  std::vector<long long> roff(P + 1, 0);
  for (int p = 0; p < P; ++p) {
    const bie_geometry& g = b.geoms[p];
    const std::string who = "problem " + std::to_string(p) + ": ";
    if (g.n_bodies < 1) return fail(ctx, BIE_ERR_INVALID, who + "n_bodies must be >= 1");
    if (!g.body_start || !g.x || !g.y || !g.dx || !g.dy || !g.ddx || !g.ddy)
      return fail(ctx, BIE_ERR_INVALID, who + "a geometry array is NULL");
    if (!b.loads[p] || !b.outs[p]) return fail(ctx, BIE_ERR_INVALID, who + "a load or output is NULL");
    if (int rc = check_local(ctx, {g.body_start, g.x, g.y, g.dx, g.dy, g.ddx, g.ddy, g.interior_pt, b.loads[p],
                                   b.outs[p]}, (who + "an array").c_str()))
      return rc;
    if (p > 0 && (g.interior_pt != nullptr) != has_ipt)
      return fail(ctx, BIE_ERR_INVALID, "batch: interior points for all problems or for none");
    has_ipt = g.interior_pt != nullptr;
    roff[p + 1] = roff[p] + g.n_bodies + 1;
    if (roff[p + 1] > 0x3fffffffLL) return fail(ctx, BIE_ERR_INVALID, "batch: too many bodies");
  }
  std::vector<int> raw(roff[P]);
  std::vector<CopySeg> segs;
  std::vector<int> on_device;
  for (int p = 0; p < P; ++p) {
    const bie_geometry& g = b.geoms[p];
    if (is_device_ptr(g.body_start)) {
      segs.push_back(CopySeg{g.body_start, nullptr, g.n_bodies + 1});
      on_device.push_back(p);
    } else {
      memcpy(raw.data() + roff[p], g.body_start, (g.n_bodies + 1) * sizeof(int));
    }
  }
  if (!segs.empty()) {
    DeviceGuard dg(ctx->device);
    int* d = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&d), roff[P] * sizeof(int), s));
    for (size_t i = 0; i < segs.size(); ++i) segs[i].dst = d + roff[on_device[i]];
    std::vector<int> tmp(roff[P]);
    cudaError_t e = gather_segments(segs, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.data(), d, roff[P] * sizeof(int), cudaMemcpyDeviceToHost, s);
    const cudaError_t f = cudaFreeAsync(d, s);  // on every path
    CK(e);
    CK(f);
    CK(cudaStreamSynchronize(s));
    for (int p : on_device) std::copy(tmp.begin() + roff[p], tmp.begin() + roff[p + 1], raw.begin() + roff[p]);
  }
  bs.assign(1, 0);
  pb.assign(1, 0);
  for (int p = 0; p < P; ++p) {
    const int* q = raw.data() + roff[p];
    const int Np = b.geoms[p].n_bodies;
    const std::string who = "problem " + std::to_string(p) + ": ";
    if (q[0] != 0) return fail(ctx, BIE_ERR_INVALID, who + "body_start[0] must be 0");
    for (int i = 0; i < Np; ++i)
      if (q[i + 1] - q[i] < 8)
        return fail(ctx, BIE_ERR_INVALID, who + "body " + std::to_string(i) + " has fewer than 8 nodes");
    const int off = bs.back();
    if ((long long)off + q[Np] > 0x3fffffffLL) return fail(ctx, BIE_ERR_INVALID, "batch: too many nodes");
    for (int i = 1; i <= Np; ++i) bs.push_back(off + q[i]);
    pb.push_back(pb.back() + Np);
  }
  return BIE_OK;
}

int check_inside(bie_ctx* ctx, const Work& w, cudaStream_t s) {
  std::vector<double> wind(w.g.N);
  CK(cudaMemcpyAsync(wind.data(), w.g.wind, w.g.N * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int i = 0; i < w.g.N; ++i)
    if (!(fabs(wind[i] - 1.0) < 0.5))
      return fail(ctx, BIE_ERR_OUTSIDE,
                  "interior point of body " + std::to_string(i) + " is not inside it (winding number " +
                      std::to_string(wind[i]) + "); is the curve counter-clockwise?");
  return BIE_OK;
}

cudaEvent_t take_event(bie_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Accumulate finished timings; with wait, block until all have finished.
void resolve_timings(bie_ctx* ctx, bool wait) {
  std::vector<bie_ctx::Timing> keep;
  for (auto& t : ctx->pending) {
    if (!wait && cudaEventQuery(t.b) != cudaSuccess) {
      cudaGetLastError();
      keep.push_back(t);
      continue;
    }
    if (wait) cudaEventSynchronize(t.b);
    if (t.valid) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
        ctx->counters.launches[t.prec][t.kind] += 1;
        ctx->counters.ms[t.prec][t.kind] += ms;
        ctx->counters.pairs[t.prec][t.kind] += t.pairs;
      } else {
        cudaGetLastError();
      }
    }
    ctx->pool.push_back(t.a);
    ctx->pool.push_back(t.b);
  }
  ctx->pending.swap(keep);
}

// Pair sum with optional event timing.  valid = false marks a launch inside a
// GMRES chunk whose validity is known only after the next state read.
cudaError_t timed_pair_sum(bie_ctx* ctx, const Geo& g, int kind, int prec, const PairPlan& p, VecRef v,
                           const double* sscale, double* partial, const int* stop, bool valid,
                           cudaStream_t s) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (ctx->prof) {
    a = take_event(ctx);
    b = take_event(ctx);
    if (a && b) cudaEventRecord(a, s);
  }
  cudaError_t e = pair_sum(g, kind, prec, p, v, sscale, partial, stop, s);
  if (a && b) {
    cudaEventRecord(b, s);
    ctx->pending.push_back({a, b, prec, kind, g.pairs > 0.0 ? g.pairs : (double)g.M * (double)(g.M - 1), valid});
  }
  return e;
}

// The operator (1/2 I + K + L) on sqrt(w)-scaled vectors, in FP64 or FP32 pair sums.
// alpha = 0: the paper's completion; alpha > 0: weighted per body (inner solves).
// fmm_p > 0: the pair sums by the FMM of that order instead of direct sums.
struct Op {
  bie_ctx* ctx;
  const Work* w;
  int prec;
  double alpha = 0.0;
  int fmm_p = 0;
  bool precond = false;  // GMRES on A P with the right block-Jacobi preconditioner P
  bool skip_stopped = false;  // batched GMRES iteration: no pair sums for stopped problems
  // out = A in (the preconditioner is applied by the GMRES driver)
  cudaError_t apply(VecRef in, VecRef out, const int* stop, cudaStream_t s, bool valid = true) const {
    if (skip_stopped && w->seg.P > 1 && fmm_p == 0) {
      Geo g = w->g;
      g.ps = w->ps;
      g.bprob = w->bprob;
      g.jstep = &w->st->j;
      const PairPlan& p = prec == 0 ? w->plan64 : (prec == 1 ? w->plan32 : w->planff);
      cudaError_t e = timed_pair_sum(ctx, g, w->kind, prec, p, in, w->g.sw, w->partial, stop, valid, s);
      if (e != cudaSuccess) return e;
      return epilogue(w->g, w->kind, p, in, w->partial, 1, 1, 1.0, out, stop, s, alpha, prec == 1, prec == 1);
    }
    if (fmm_p > 0) {
      const PairPlan one = uniform_plan(1, w->g.M);
      cudaError_t e = fmm_pair_sum(ctx->fmm, w->g, w->kind, fmm_p, in, w->g.sw, w->partial, stop, s, prec);
      if (e != cudaSuccess) return e;
      return epilogue(w->g, w->kind, one, in, w->partial, 1, 1, 1.0, out, stop, s, alpha, false, prec == 1);
    }
    const PairPlan& p = prec == 0 ? w->plan64 : (prec == 1 ? w->plan32 : w->planff);
    cudaError_t e = timed_pair_sum(ctx, w->g, w->kind, prec, p, in, w->g.sw, w->partial, stop, valid, s);
    if (e != cudaSuccess) return e;
    return epilogue(w->g, w->kind, p, in, w->partial, 1, 1, 1.0, out, stop, s, alpha, prec == 1, prec == 1);
  }
};

struct KrylovResult {
  int iters = 0, matvecs = 0, matvecs64 = 0;
  double res = 0.0, bnorm = 0.0;
  bool converged = false;
  std::vector<double> prel;  // batched GMRES: every problem's relative residual
};

int read_state(bie_ctx* ctx, const Work& w, cudaStream_t s) {
  CK(cudaMemcpyAsync(ctx->h_state, w.st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return BIE_OK;
}

// Restarted GMRES from x = 0 on A x = b until ||b - A x|| <= tol_rel ||b||.
// Each cycle minimises over x + span(V) with V_0 = r/||r||, so gmres_update
// adds V y into x and a restart only needs the explicit residual.  With
// verify, convergence is confirmed by an explicit residual of the FP64 operator.
// One Arnoldi iteration: w = A v_j, CGS2 against V_0..V_j, Givens, v_{j+1}.
// Every kernel reads j from the device state, so the same launches (or the
// same captured graph) serve every iteration.
int launch_iteration(bie_ctx* ctx, Work& w, const Op& op, cudaStream_t s) {
  const long long n = w.n, ld = w.ld;
  const VecRef vj{w.V, ld, &w.st->j, 0}, vj1{w.V, ld, &w.st->j, 1};
  // w = A v_j, or A z_j with z_j = P v_j left in zbuf by the previous step
  Op it = op;
  it.skip_stopped = true;
  CK(it.apply(op.precond ? vec(w.zbuf) : vj, vj1, &w.st->stop, s, false));
  ArnoldiArgs a{w.V,        ld,       n,      w.st,      w.arn, w.H, w.cs, w.sn, w.gv, w.g,
                w.kind,     w.bj_off, op.precond ? w.bj_blocks : nullptr, w.zbuf};
  a.bj64 = op.prec == 0;  // FP64 GMRES: the preconditioner applied in FP64 arithmetic
  if (w.seg.P > 1) {
    CK(arnoldi_seg(a, w.seg, w.seg_grid, s));
  } else {
    // the FP32 inner solves: CGS2 in FP32 against the FP32 basis
    if (op.prec == 1 && w.VF) a.vf = w.VF;
    CK(arnoldi(a, arnoldi_grid(n, a.vf != nullptr, w.g.N), s));
  }
  return BIE_OK;
}

bool capturable(cudaStream_t s) {
  return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

// The iteration as a CUDA graph (built once per workspace layout and operator;
// not while pair-sum timing is on, whose events are per launch).  nullptr if
// the stream cannot be captured.
bie_ctx::IterGraph* iteration_graph(bie_ctx* ctx, Work& w, const Op& op, cudaStream_t s) {
  if (ctx->prof || !capturable(s) || barrier_fault_armed()) return nullptr;
  const PairPlan& p = op.prec == 0 ? w.plan64 : (op.prec == 1 ? w.plan32 : w.planff);
  long long alpha_bits;
  memcpy(&alpha_bits, &op.alpha, sizeof(alpha_bits));
  // an FMM application's captured launches depend on the tree (buffers, level
  // count, bounding square), which a later setup may rebuild or reallocate
  long long fsig[2] = {0, 0};
  if (op.fmm_p > 0) fmm_signature(ctx->fmm, fsig);
  const long long key[12] = {(long long)(uintptr_t)ctx->ws, (long long)ctx->ws_size, w.g.N, w.g.M,
                             w.kind + 4LL * w.seg.P, w.m, op.prec * 1000 + op.fmm_p + (op.precond ? 500 : 0), alpha_bits,
                             (p.S * 1000003LL + p.chunk) * 1000003LL + p.S1 * 4099LL + p.chunk2 * 2 + p.sym,
                             w.grid + 1000003LL * w.seg.nitem, fsig[0], fsig[1]};
  for (auto& gi : ctx->graphs)
    if (memcmp(gi.key, key, sizeof(key)) == 0) return &gi;
  auto keep = [&](cudaGraphExec_t exec, long long kernels) {
    if (ctx->graphs.size() >= 4) {
      cudaGraphExecDestroy(ctx->graphs.front().exec);
      ctx->graphs.erase(ctx->graphs.begin());
    }
    bie_ctx::IterGraph gi;
    memcpy(gi.key, key, sizeof(key));
    gi.exec = exec;
    gi.kernels = kernels;
    gi.last_cycle = 0;
    ctx->graphs.push_back(gi);
    return &ctx->graphs.back();
  };
  const long long before = thread_launches();
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const int rc = launch_iteration(ctx, w, op, s);
  const cudaError_t e = cudaStreamEndCapture(s, &graph);
  const long long kernels = thread_launches() - before;
  note_launches((int)-kernels);  // captured, not launched
  cudaGraphExec_t exec = nullptr;
  if (rc != BIE_OK || e != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return nullptr;
  }
  cudaGraphDestroy(graph);
  return keep(exec, kernels);
}

// One GMRES cycle: iterations launched in chunks (graph replays where the
// stream can be captured) with a state read after each chunk.  Iterations
// launched after the one that stops the cycle return at once; to launch few
// of them without reading the state more often, the first chunk is as long as
// the last cycle replayed from the same graph (the cycles of a refinement, and
// the solves of one shape, take similar counts), the later ones 2, 4, 8, 16.
int run_cycle(bie_ctx* ctx, Work& w, const Op& op, cudaStream_t s) {
  int rc;
  const int start = ctx->h_state->iters;
  int iters_before = start;
  bie_ctx::IterGraph* graph = iteration_graph(ctx, w, op, s);
  ctx->graph_replay = graph ? 1 : 0;
  int chunk = graph && graph->last_cycle > 0 ? graph->last_cycle : 4, next = graph && graph->last_cycle > 0 ? 2 : 8;
  for (;;) {
    const size_t mark = ctx->pending.size();
    for (int it = 0; it < chunk; ++it) {
      if (graph) {
        CK(cudaGraphLaunch(graph->exec, s));
        note_launches((int)graph->kernels);
      } else if ((rc = launch_iteration(ctx, w, op, s))) {
        return rc;
      }
    }
    if ((rc = read_state(ctx, w, s))) return rc;
    if (ctx->h_state->error)
      return fail(ctx, BIE_ERR_TIMEOUT, "a grid barrier of the Arnoldi step timed out (a CTA never arrived)");
    const int done = ctx->h_state->iters - iters_before;
    for (size_t k = mark; k < ctx->pending.size(); ++k) ctx->pending[k].valid = (int)(k - mark) < done;
    resolve_timings(ctx, false);
    iters_before = ctx->h_state->iters;
    if (ctx->h_state->stop) {
      if (graph) graph->last_cycle = std::max(1, std::min(ctx->h_state->iters - start, w.m));
      return BIE_OK;
    }
    chunk = next;
    next = std::min(next * 2, 16);
  }
}

int gmres(bie_ctx* ctx, Work& w, const Op& op, const double* b, double* x, double tol_rel, int maxit,
          bool verify, KrylovResult& out, cudaStream_t s) {
  const long long n = w.n, ld = w.ld;
  KState init;
  memset(&init, 0, sizeof(init));
  init.scratch[0] = tol_rel;
  init.pad[0] = 1;  // k_residual sets tol_abs = tol_rel * ||b|| on the first call
  init.maxit = maxit;
  init.m = w.m;
  *ctx->h_state = init;
  CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(KState), cudaMemcpyHostToDevice, s));
  CK(fill0(x, n, s));
  CK(residual_start(b, nullptr, w.rin, w.V, n, w.st, w.part, w.gv, 1, w.grid, s));
  if (op.precond) CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.V), w.zbuf, &w.st->stop, w.bj_max_nb, s, op.prec == 0));
  Op rop = verify ? Op{ctx, &w, 0} : op;
  rop.precond = false;  // residuals of x itself (x = P y is kept in original variables)
  int rc;
  for (;;) {
    if ((rc = run_cycle(ctx, w, op, s))) return rc;
    const KState h = *ctx->h_state;
    out.bnorm = h.scratch[1];
    out.iters = h.iters;
    if (h.j > 0) {
      if (op.precond) {  // x += P (V y)
        CK(fill0(w.ytmp, n, s));
        CK(gmres_update(w.V, ld, n, w.st, w.H, w.gv, w.yv, w.ytmp, w.grid, s));
        CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.ytmp), w.zbuf, nullptr, w.bj_max_nb, s, op.prec == 0));
        CK(axpy(x, w.zbuf, n, s));
      } else {
        CK(gmres_update(w.V, ld, n, w.st, w.H, w.gv, w.yv, x, w.grid, s));
      }
    }
    out.matvecs += h.j;
    if (h.j == 0) {  // nothing to do: b is (numerically) zero or the cap is reached
      out.res = h.rnorm;
      out.converged = h.rnorm <= h.tol_abs;
      return BIE_OK;
    }
    if (!verify && (h.res <= h.tol_abs || h.iters >= h.maxit)) {
      out.res = h.res;
      out.converged = h.res <= h.tol_abs;
      return BIE_OK;
    }
    // explicit residual; opens the next cycle unless converged or capped
    CK(rop.apply(vec(x), vec(w.ytmp), nullptr, s));
    if (verify) out.matvecs64 += 1; else out.matvecs += 1;
    CK(residual_start(b, w.ytmp, w.rin, w.V, n, w.st, w.part, w.gv, 1, w.grid, s));
    if (op.precond) CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.V), w.zbuf, &w.st->stop, w.bj_max_nb, s, op.prec == 0));
    if ((rc = read_state(ctx, w, s))) return rc;
    const KState& h2 = *ctx->h_state;
    if (h2.rnorm <= h2.tol_abs || h2.iters >= h2.maxit) {
      out.res = h2.rnorm;
      out.converged = h2.rnorm <= h2.tol_abs;
      return BIE_OK;
    }
  }
}

// Batched restarted GMRES: the same iteration with one Krylov space per
// problem (the problems advance in lockstep; each stops at its own
// tolerance, tol_rel ||b_p||).  out.res and out.bnorm are those of the problem
// with the largest relative residual (true residuals with verify).
int gmres_seg(bie_ctx* ctx, Work& w, const Op& op, const double* b, double* x, double tol_rel, int maxit,
              bool verify, KrylovResult& out, cudaStream_t s) {
  const long long n = w.n, ld = w.ld;
  KState init;
  memset(&init, 0, sizeof(init));
  init.scratch[0] = tol_rel;
  init.pad[0] = 1;  // k_residual_seg sets every problem's tolerance on the first call
  init.maxit = maxit;
  init.m = w.m;
  *ctx->h_state = init;
  CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(KState), cudaMemcpyHostToDevice, s));
  CK(fill0(x, n, s));
  CK(residual_start_seg(b, nullptr, w.rin, w.V, w.st, w.seg, w.gv, w.m, s));
  if (op.precond) CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.V), w.zbuf, &w.st->stop, w.bj_max_nb, s, op.prec == 0));
  Op rop = verify ? Op{ctx, &w, 0} : op;
  rop.precond = false;
  auto worst = [&](bool converged) -> int {
    std::vector<PState> ps(w.seg.P);
    CK(cudaMemcpyAsync(ps.data(), w.ps, ps.size() * sizeof(PState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rel = -1.0;
    out.prel.clear();
    for (const PState& q : ps) {
      const double r = verify ? q.rnorm : q.res;
      const double e = q.bnorm > 0.0 ? r / q.bnorm : 0.0;
      out.prel.push_back(e);
      if (e > rel) {
        rel = e;
        out.res = r;
        out.bnorm = q.bnorm;
      }
    }
    out.converged = converged;
    return BIE_OK;
  };
  int rc;
  for (;;) {
    if ((rc = run_cycle(ctx, w, op, s))) return rc;
    const KState h = *ctx->h_state;
    out.iters = h.iters;
    if (h.j > 0) {
      if (op.precond) {  // x += P (V y)
        CK(fill0(w.ytmp, n, s));
        CK(gmres_update_seg(w.V, ld, w.st, w.seg, w.H, w.gv, w.yv, w.ytmp, w.m, w.max_plen, s));
        CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.ytmp), w.zbuf, nullptr, w.bj_max_nb, s, op.prec == 0));
        CK(axpy(x, w.zbuf, n, s));
      } else {
        CK(gmres_update_seg(w.V, ld, w.st, w.seg, w.H, w.gv, w.yv, x, w.m, w.max_plen, s));
      }
    }
    out.matvecs += h.j;
    if (h.j == 0) return worst(h.nactive == 0);
    if (!verify && (h.nactive == 0 || h.iters >= h.maxit)) return worst(h.nactive == 0);
    // explicit residual; opens the next cycle for the problems above tolerance
    CK(rop.apply(vec(x), vec(w.ytmp), nullptr, s));
    if (verify) out.matvecs64 += 1; else out.matvecs += 1;
    CK(residual_start_seg(b, w.ytmp, w.rin, w.V, w.st, w.seg, w.gv, w.m, s));
    if (op.precond) CK(bj_apply(w.g, w.kind, w.bj_off, w.bj_blocks, vec(w.V), w.zbuf, &w.st->stop, w.bj_max_nb, s, op.prec == 0));
    if ((rc = read_state(ctx, w, s))) return rc;
    const KState& h2 = *ctx->h_state;
    if (h2.nactive == 0 || h2.iters >= h2.maxit) return worst(h2.nactive == 0);
  }
}

int copy_out(bie_ctx* ctx, double* dst, const double* src, size_t count, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, s));
  return BIE_OK;
}

void fill_opts(const bie_opts* o, bie_opts& r) {
  r.tol = 1e-12;
  r.max_iter = 500;
  r.restart = 50;
  r.precision = BIE_PREC_FP64;
  r.formulation = 0;
  r.max_refine = 8;
  r.inner_tol = 1e-6;
  r.fmm_order = 0;
  r.precond = 0;
  if (!o) return;
  if (o->tol > 0) r.tol = o->tol;
  if (o->max_iter > 0) r.max_iter = o->max_iter;
  if (o->restart > 0) r.restart = std::min(o->restart, 200);
  r.precision = o->precision;
  r.formulation = o->formulation;
  r.precond = o->precond;
  if (o->max_refine > 0) r.max_refine = o->max_refine;
  if (o->inner_tol > 0) r.inner_tol = o->inner_tol;
  r.fmm_order = o->fmm_order;
}

int solve_common(bie_ctx* ctx, const bie_geometry* geom, int kind, const double* load, double* out,
                 double* density, const bie_opts* opts_in, bie_info* info, cudaStream_t s,
                 const BatchIn* batch = nullptr) {
  std::vector<int> bs, pb;
  bool has_ipt = false;
  int rc;
  if (batch) {
    if (!ctx) return BIE_ERR_INVALID;
    if (batch->P < 1 || batch->P > 65535 || !batch->geoms || !batch->loads || !batch->outs)
      return fail(ctx, BIE_ERR_INVALID, "batch: count outside 1..65535 or a NULL array");
    if (density) return fail(ctx, BIE_ERR_INVALID, "batch: no density output");
    if ((rc = validate_batch(ctx, *batch, bs, pb, has_ipt, s))) return rc;
  } else {
    if ((rc = validate(ctx, geom, bs))) return rc;
    if (!load || !out) return fail(ctx, BIE_ERR_INVALID, "load or output pointer is NULL");
    if ((rc = check_local(ctx, {load, out, density}, "a load, output or density array"))) return rc;
    has_ipt = geom->interior_pt != nullptr;
  }
  bie_opts o;
  fill_opts(opts_in, o);
  if (o.precision != BIE_PREC_FP64 && o.precision != BIE_PREC_MIXED && o.precision != BIE_PREC_MIXED_FF)
    return fail(ctx, BIE_ERR_INVALID, "precision must be BIE_PREC_FP64, BIE_PREC_MIXED or BIE_PREC_MIXED_FF");
  if (o.formulation != 0 && o.formulation != 1) return fail(ctx, BIE_ERR_INVALID, "formulation must be 0 or 1");
  if (o.precond != 0 && o.precond != 1) return fail(ctx, BIE_ERR_INVALID, "precond must be 0 or 1");
  if (o.fmm_order != 0 && (std::abs(o.fmm_order) < 2 || std::abs(o.fmm_order) > 64))
    return fail(ctx, BIE_ERR_INVALID, "fmm_order must be 0, in 2..64 or in -64..-2");
  if (o.fmm_order < 0 && o.precision == BIE_PREC_FP64)
    return fail(ctx, BIE_ERR_INVALID, "fmm_order < 0 (FMM residuals only) needs a mixed precision");
  if (batch && o.fmm_order != 0) return fail(ctx, BIE_ERR_INVALID, "batch: direct pair sums only (fmm_order 0)");
  DeviceGuard dg(ctx->device);
  const int N = (int)bs.size() - 1, M = bs[N];
  const int P = batch ? batch->P : 1;
  const int nload = kind == 0 ? N : 3 * N;
  Work w;
  // batches of small problems: one persistent launch, one CTA per problem
  // running the whole float-float refinement (no host round trip, no
  // preconditioner)
  int small_nodes = 0;
  bool small = false;
  if (batch && small_batch_path() && o.precision == BIE_PREC_MIXED_FF && o.fmm_order == 0) {
    int max_bodies = 0;
    for (int p = 0; p < P; ++p) {
      small_nodes = std::max(small_nodes, bs[pb[p + 1]] - bs[pb[p]]);
      max_bodies = std::max(max_bodies, pb[p + 1] - pb[p]);
    }
    small = small_batch_eligible(small_nodes, max_bodies, o.restart);
  }
  const bool use_bj = o.precond == 0 && !small;
  const long long bjf = use_bj ? bj_block_floats(bs.data(), N, kind) : 0;
  Arena sz{nullptr};
  carve(sz, w, N, M, kind, o.restart, true, true, has_ipt, true, false, bjf, batch ? P : 0, bs.data(), pb.data());
  if ((rc = ensure_ws(ctx, sz.off, s))) return rc;
  Arena ar{ctx->ws};
  carve(ar, w, N, M, kind, o.restart, true, true, has_ipt, true, false, bjf, batch ? P : 0, bs.data(), pb.data());
  if (batch) {
    if ((rc = batch_setup(ctx, *batch, bs, pb, has_ipt, w, s))) return rc;
  } else if ((rc = setup(ctx, geom, bs, w, s))) {
    return rc;
  }
  if (bjf > 0) {
    for (int i = 0; i < N; ++i) w.bj_max_nb = std::max(w.bj_max_nb, (bs[i + 1] - bs[i]) * (kind + 1));
  }
  const double* dload = w.load;
  if (!batch && (rc = stage_in(ctx, load, w.load, nload, &dload, s))) return rc;
  if ((rc = check_inside(ctx, w, s))) return rc;
  // fmm_order > 0: FMM pair sums everywhere; < 0: for the residuals and outputs only
  const int p_res = std::abs(o.fmm_order);
  const FmmSchedule fsched = p_res > 0 ? fmm_schedule(M, kind, p_res) : FmmSchedule{0, 0};
  const int p_in = o.fmm_order > 0 ? fsched.inner_order : 0;
  if (p_res > 0) {
    const int orders[2] = {p_res, std::max(2, p_in)};
    if ((rc = fmm_setup(ctx->fmm, w.g, kind, orders, o.fmm_order > 0 ? 2 : 1, s, ctx->err, fsched.leaf_nodes)))
      return rc;
  }
  // the block of the operator GMRES iterates on: the paper's completion (FP64
  // GMRES) or the weighted one of the inner solves
  if (bjf > 0)
    CK(bj_setup(w.g, kind, o.precision == BIE_PREC_FP64 ? 0.0 : kInnerCompletionWeight, bs.data(), w.bj_off,
                w.bj_pairs, w.bj_blocks, w.bj_fallbacks, s));

  const long long n = w.n;
  // right-hand side (scaled by sqrt(w))
  if (o.formulation == 0) {
    CK(total_density_rhs(w.g, kind, dload, w.f, s));
  } else {
    CK(incident_density_scaled(w.g, kind, dload, w.rin, s));
    CK(timed_pair_sum(ctx, w.g, kind, 0, w.plan64, vec(w.rin), w.g.sw, w.partial, nullptr, true, s));
    CK(epilogue(w.g, kind, w.plan64, vec(w.rin), w.partial, 1, 0, -1.0, vec(w.f), nullptr, s));
  }
  // a batch: every problem's right-hand side scaled to unit norm and the
  // tolerance made absolute, so that each problem's own relative residual is
  // at most the combined residual (the solution is scaled back below)
  double fnorm_batch = 1.0;
  const double tol_user = o.tol;
  if (batch) {
    CK(batch_normalize(P, w.pnode, w.f, w.pscale, s));
    KState init;
    memset(&init, 0, sizeof(init));
    *ctx->h_state = init;
    CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(KState), cudaMemcpyHostToDevice, s));
    CK(residual_start(w.f, nullptr, w.ytmp, w.V, n, w.st, w.part, w.gv, 0, w.grid, s));
    if ((rc = read_state(ctx, w, s))) return rc;
    fnorm_batch = ctx->h_state->rnorm;
    if (fnorm_batch > 0.0) o.tol /= fnorm_batch;
  }
  // inner FP32 solves use the completion weighted per body (weight 1/|Gamma_i|):
  // same solution, no outlier eigenvalue per body in the Krylov spectrum
  const int fres = p_res, fin = o.fmm_order > 0 ? std::max(2, p_in) : 0;
  const Op op64{ctx, &w, 0, 0.0, fres, o.precision == BIE_PREC_FP64 && bjf > 0},
      op32{ctx, &w, 1, kInnerCompletionWeight, fin, bjf > 0};
  // refinement residual: FP64, or float-float for BIE_PREC_MIXED_FF (direct sums),
  // or the FMM of the full order
  const Op opres{ctx, &w, o.precision == BIE_PREC_MIXED_FF ? 2 : 0, 0.0, fres};
  int m64 = o.formulation == 1 ? 1 : 0, m32 = 0, mff = 0, iters = 0, refs = 0;
  double relres = 0.0, eps32_report = 0.0;
  bool converged = false, relres_per_problem = false;
  std::vector<double> prob_rel;  // batched: every problem's relative residual
  // GMRES on one system, or (several problems) one Krylov space per problem
  auto krylov = [&](const Op& op, const double* b, double* x, double tol_rel, int maxit, bool verify,
                    KrylovResult& kr) -> int {
    return w.seg.P > 1 ? gmres_seg(ctx, w, op, b, x, tol_rel, maxit, verify, kr, s)
                       : gmres(ctx, w, op, b, x, tol_rel, maxit, verify, kr, s);
  };
  std::vector<SmallInfo> sinfo;
  {
    if (small) {
      CK(small_batch_solve(w.g, kind, P, w.pbody, w.pnode, w.f, w.xs, w.r, w.d, w.rc, w.rin, w.ytmp, w.V, w.ld, w.m,
                           tol_user, o.inner_tol, o.max_refine, o.max_iter, small_nodes, w.sinfo, s));
      sinfo.resize(P);
      CK(cudaMemcpyAsync(sinfo.data(), w.sinfo, P * sizeof(SmallInfo), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      converged = true;
      for (const SmallInfo& q : sinfo) {
        iters = std::max(iters, q.iters);
        refs = std::max(refs, q.refinements);
        m32 += q.matvecs32;
        mff += q.matvecsff;
        eps32_report = std::max(eps32_report, q.fp32_error);
        prob_rel.push_back(q.rel_residual);
        relres = std::max(relres, q.rel_residual);
        converged = converged && q.rel_residual <= tol_user;
      }
      relres_per_problem = true;
    }
  }
  if (small) {
    // solved above
  } else if (o.precision == BIE_PREC_FP64) {
    KrylovResult kr;
    // batched: every problem to the relative tolerance on its own right-hand side
    if ((rc = krylov(op64, w.f, w.xs, w.seg.P > 1 ? tol_user : o.tol, o.max_iter, true, kr))) return rc;
    m64 += kr.matvecs + kr.matvecs64;
    iters = kr.iters;
    relres = kr.bnorm > 0 ? kr.res / kr.bnorm : 0.0;
    relres_per_problem = w.seg.P > 1;
    converged = kr.converged;
    prob_rel = kr.prel;
  } else {
    // FP64 iterative refinement: x += A32^{-1}(f - A64 x)
    CK(fill0(w.xs, n, s));
    CK(cudaMemcpyAsync(w.r, w.f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // ||f||
    {
      KState init;
      memset(&init, 0, sizeof(init));
      *ctx->h_state = init;
      CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(KState), cudaMemcpyHostToDevice, s));
      CK(residual_start(w.f, nullptr, w.ytmp, w.V, n, w.st, w.part, w.gv, 0, w.grid, s));
      if ((rc = read_state(ctx, w, s))) return rc;
    }
    const double fnorm = ctx->h_state->rnorm;
    double rnorm = fnorm;
    int remaining = o.max_iter;
    converged = fnorm == 0.0;
    // ||a - b|| (b may be NULL) into out, through the residual kernel
    auto norm_of = [&](const double* a, const double* b, double* out) -> int {
      KState init;
      memset(&init, 0, sizeof(init));
      *ctx->h_state = init;
      CK(cudaMemcpyAsync(w.st, ctx->h_state, sizeof(KState), cudaMemcpyHostToDevice, s));
      CK(residual_start(a, b, out, w.V, n, w.st, w.part, w.gv, 0, w.grid, s));
      return read_state(ctx, w, s);
    };
    // Float-float refinement updates the residual after the first true one:
    // r -= A32 d, with the FP32 operator's relative error eps32 measured on this
    // geometry (A32 x against A_ff x at the first step) and the accumulated
    // bound 3 eps32 sum ||A32 d|| added to ||r|| before comparing with tol.
    const bool recursive = o.precision == BIE_PREC_MIXED_FF && o.fmm_order <= 0;
    const Op op32p{ctx, &w, 1, 0.0, fin};  // FP32 pair sums (or FP32 FMM), the paper's completion
    double eps32 = -1.0, bound = 0.0;
    bool true_residual = true;
    // batched (one Krylov space per problem): every problem's own residual
    // (right-hand sides of unit norm) against the tolerance, and a problem
    // already below it sits out the next inner solve
    const bool per_problem = w.seg.P > 1;
    double worst = 0.0;
    std::vector<double> pn_host(per_problem ? w.seg.P : 0);
    auto problem_norms = [&]() -> int {
      CK(seg_norms(w.seg.P, w.pnode, w.r, w.pnorm, s));
      CK(cudaMemcpyAsync(pn_host.data(), w.pnorm, pn_host.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      worst = 0.0;
      for (double v : pn_host) worst = std::max(worst, v);
      return BIE_OK;
    };
    if (per_problem && (rc = problem_norms())) return rc;
    while (!converged && refs < o.max_refine && remaining > 0) {
      KrylovResult kr;
      CK(consistent_rhs(w.g, kind, kInnerCompletionWeight, w.r, w.rc, s));
      if (per_problem && tol_user - bound > 0.0)
        CK(seg_zero_below(w.seg.P, w.pnode, w.pnorm, tol_user - bound, w.rc, s));
      if ((rc = krylov(op32, w.rc, w.d, o.inner_tol, remaining, false, kr))) return rc;
      iters += kr.iters;
      m32 += kr.matvecs;
      remaining -= kr.iters;
      refs += 1;
      CK(axpy(w.xs, w.d, n, s));
      if (recursive && !true_residual && eps32 >= 0.0) {
        CK(op32p.apply(vec(w.d), vec(w.ytmp), nullptr, s));
        m32 += 1;
        if ((rc = norm_of(w.ytmp, nullptr, w.rin))) return rc;
        bound += 3.0 * eps32 * ctx->h_state->rnorm;
        if ((rc = norm_of(w.r, w.ytmp, w.r))) return rc;
        rnorm = ctx->h_state->rnorm + bound;
        // once the bound eats half the tolerance, go back to a true residual
        if (bound > 0.5 * o.tol * fnorm) true_residual = true;
      } else {
        CK(opres.apply(vec(w.xs), vec(w.ytmp), nullptr, s));
        if (opres.prec == 0 || opres.fmm_p > 0) m64 += 1; else mff += 1;
        if ((rc = norm_of(w.f, w.ytmp, w.r))) return rc;
        rnorm = ctx->h_state->rnorm;
        bound = 0.0;
        if (eps32 < 0.0) {
          // eps32 = ||A x - A32 x|| / ||A x||, A the residual operator (reported; the
          // float-float refinement's residual update bound uses it)
          CK(op32p.apply(vec(w.xs), vec(w.rin), nullptr, s));
          m32 += 1;
          if ((rc = norm_of(w.ytmp, w.rin, w.rc))) return rc;
          const double diff = ctx->h_state->rnorm;
          if ((rc = norm_of(w.ytmp, nullptr, w.rc))) return rc;
          const double ref = ctx->h_state->rnorm;
          eps32 = ref > 0.0 ? diff / ref : 0.0;
        }
        true_residual = !recursive;
      }
      if (per_problem) {
        if ((rc = problem_norms())) return rc;
        converged = worst + bound <= tol_user;
      } else {
        converged = rnorm <= o.tol * fnorm;
      }
      if (kr.iters == 0) break;
    }
    relres = fnorm > 0 ? rnorm / fnorm : 0.0;
    if (per_problem) {
      relres = worst + bound;  // the largest relative residual of any problem (unit right-hand sides)
      relres_per_problem = true;
      for (double v : pn_host) prob_rel.push_back(v + bound);
    }
    eps32_report = eps32 > 0.0 ? eps32 : 0.0;
  }
  if (batch) {
    CK(batch_unscale(P, w.pnode, w.pscale, w.xs, s));
    // the combined residual of the unit right-hand sides bounds every problem's
    // relative residual
    if (!relres_per_problem) relres *= fnorm_batch;
  }
  // total density (scaled): nu = x (total form) or mu + sigma (paper form)
  double* v = w.xs;
  if (o.formulation == 1) {
    CK(incident_density_scaled(w.g, kind, dload, w.rin, s));
    CK(axpy(w.xs, w.rin, n, s));
  }
  if (o.fmm_order != 0) {
    CK(fmm_output(ctx->fmm, w.g, kind, p_res, v, w.outpart, s, o.precision == BIE_PREC_MIXED_FF));
    CK(finalize_output(w.g, kind, v, dload, w.outpart, 1, w.outv, w.cres, s));
  } else {
    CK(evaluate_output(w.g, kind, v, dload, w.outpart, w.P, w.outv, w.cres, s));
  }
  if (density) {
    CK(unscale(w.g, kind, v, w.ytmp, s));
    if ((rc = copy_out(ctx, density, w.ytmp, n, s))) return rc;
  }
  if (batch) {
    // device outputs scattered by one kernel, host outputs from one read-back
    std::vector<CopySeg> segs;
    std::vector<int> on_host;
    const int per = kind == 0 ? 1 : 3;
    for (int p = 0; p < P; ++p) {
      const long long nl = (long long)(pb[p + 1] - pb[p]) * per;
      if (is_device_ptr(batch->outs[p]))
        segs.push_back(CopySeg{w.outv + (long long)pb[p] * per, batch->outs[p], 2 * nl});
      else
        on_host.push_back(p);
    }
    CK(gather_segments(segs, s));
    if (!on_host.empty()) {
      std::vector<double> h(nload);
      CK(cudaMemcpyAsync(h.data(), w.outv, nload * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int p : on_host)
        memcpy(batch->outs[p], h.data() + (long long)pb[p] * per, (size_t)(pb[p + 1] - pb[p]) * per * sizeof(double));
    }
  } else if ((rc = copy_out(ctx, out, w.outv, nload, s))) {
    return rc;
  }
  // constraint residual and net load
  const int targets = kind == 0 ? N : 3 * N;
  const int P_used = o.fmm_order != 0 ? 1 : w.P;  // splits of the output sums
  const double* nl = w.outpart + (size_t)P_used * targets * (kind + 1) + N;
  CK(cudaMemcpyAsync(ctx->h_small, w.cres, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ctx->h_small + 1, nl, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  int* h_fb = reinterpret_cast<int*>(ctx->h_small + 3);
  *h_fb = 0;
  if (w.bj_fallbacks) CK(cudaMemcpyAsync(h_fb, w.bj_fallbacks, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (batch) {
    // every problem's own info and status: per-body constraint values and
    // per-problem net loads from the output kernels
    std::vector<double> cbody(N), pnet(2 * P);
    CK(cudaMemcpyAsync(cbody.data(), nl - N, N * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(pnet.data(), w.pnet, 2 * P * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (prob_rel.size() != (size_t)P) prob_rel.assign(P, relres);  // a batch of one
    int worst_status = BIE_OK;
    for (int p = 0; p < P; ++p) {
      double cmax = 0.0;
      for (int i = pb[p]; i < pb[p + 1]; ++i) cmax = std::max(cmax, cbody[i]);
      const double net = pnet[2 * p], mx = pnet[2 * p + 1];
      const int Np = pb[p + 1] - pb[p];
      int st = BIE_OK;
      if (!(prob_rel[p] <= tol_user) && !(converged && P == 1)) st = BIE_WARN_NOT_CONVERGED;
      else if (net > 1e-12 * std::max(mx, 1e-300) * std::max(1, Np)) st = BIE_WARN_NONNEUTRAL;
      if (batch->status) batch->status[p] = st;
      if (batch->infos) {
        bie_info& q = batch->infos[p];
        q.iters = iters;
        q.refinements = refs;
        q.matvecs_fp64 = m64;
        q.matvecs_fp32 = m32;
        q.matvecs_ff = mff;
        if (small) {  // the one-launch path: each problem's own counts
          q.iters = sinfo[p].iters;
          q.refinements = sinfo[p].refinements;
          q.matvecs_fp32 = sinfo[p].matvecs32;
          q.matvecs_ff = sinfo[p].matvecsff;
        }
        q.rel_residual = prob_rel[p];
        q.constraint_residual = cmax / std::max(mx, 1e-300);
        q.net_load = net;
        q.fp32_error = eps32_report;
        q.precond_fallbacks = *h_fb;  // of the whole batch
        q.graph_replay = ctx->graph_replay;
      }
      if (st == BIE_WARN_NOT_CONVERGED || (st == BIE_WARN_NONNEUTRAL && worst_status == BIE_OK)) worst_status = st;
    }
    return worst_status;
  }
  CK(cudaStreamSynchronize(s));
  const double netload = ctx->h_small[1], maxload = ctx->h_small[2];
  if (info) {
    info->iters = iters;
    info->refinements = refs;
    info->matvecs_fp64 = m64;
    info->matvecs_fp32 = m32;
    info->matvecs_ff = mff;
    info->rel_residual = relres;
    info->constraint_residual = ctx->h_small[0];
    info->net_load = netload;
    info->fp32_error = eps32_report;
    info->precond_fallbacks = *h_fb;
    info->graph_replay = ctx->graph_replay;
  }
  if (!converged) return BIE_WARN_NOT_CONVERGED;
  if (netload > 1e-12 * std::max(maxload, 1e-300) * std::max(1, N)) return BIE_WARN_NONNEUTRAL;
  return BIE_OK;
}

}  // namespace

extern "C" {

int bie_create(bie_ctx** out, int device, size_t cap) {
  if (!out) return BIE_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  bie_ctx* c = new bie_ctx();
  c->device = device;
  c->cap = cap;
  DeviceGuard dg(device);
  if (cudaMallocHost(&c->h_state, sizeof(KState)) != cudaSuccess ||
      cudaMallocHost(&c->h_small, 8 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    if (c->h_state) cudaFreeHost(c->h_state);
    delete c;
    return BIE_ERR_CUDA;
  }
  *out = c;
  return BIE_OK;
}

}  // extern "C"

namespace bie {
void release_workspace(bie_ctx* ctx, cudaStream_t s) {
  if (ctx && ctx->ws) {
    cudaFreeAsync(ctx->ws, s);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    for (auto& gi : ctx->graphs) cudaGraphExecDestroy(gi.exec);
    ctx->graphs.clear();
  }
}
}  // namespace bie

namespace bie {
size_t workspace_bytes_batch(int kind, const int* bs, int n_bodies, const int* pb, int nprob, const bie_opts* opts) {
  bie_opts o;
  fill_opts(opts, o);
  Work w;
  Arena sz{nullptr};
  const bool use_bj = o.precond == 0;
  carve(sz, w, n_bodies, bs[n_bodies], kind, o.restart, true, true, true, true, false,
        use_bj ? bj_block_floats(bs, n_bodies, kind) : 0, nprob, bs, pb);
  return sz.off;
}

size_t workspace_bytes_for(int kind, const int* body_start_host, int n_bodies, int restart) {
  const int n_nodes = body_start_host[n_bodies];
  Work w;
  Arena sz{nullptr};
  const int m = restart > 0 ? std::min(restart, 200) : 50;
  carve(sz, w, n_bodies, n_nodes, kind, m, true, true, true, true, false,
        bj_block_floats(body_start_host, n_bodies, kind));
  return sz.off;
}
}  // namespace bie

extern "C" {

int apply_operator_fmm(bie_ctx* ctx, const bie_geometry* geom, int kind, int order, const double* in, double* out,
                       void* stream) {
  return apply_operator_fmm_prec(ctx, geom, kind, order, BIE_PREC_FP64, in, out, stream);
}

int apply_operator_fmm_prec(bie_ctx* ctx, const bie_geometry* geom, int kind, int order, int precision,
                            const double* in, double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> bs;
  int rc = validate(ctx, geom, bs);
  if (rc) return rc;
  if (kind != BIE_KIND_LAPLACE && kind != BIE_KIND_STOKES) return fail(ctx, BIE_ERR_INVALID, "bad kind");
  if (order < 2 || order > 64) return fail(ctx, BIE_ERR_INVALID, "order must be in 2..64");
  if (precision != BIE_PREC_FP64 && precision != BIE_PREC_MIXED && precision != BIE_PREC_MIXED_FF)
    return fail(ctx, BIE_ERR_INVALID, "bad precision");
  if (!in || !out) return fail(ctx, BIE_ERR_INVALID, "in or out is NULL");
  if ((rc = check_local(ctx, {in, out}, "in or out"))) return rc;
  DeviceGuard dg(ctx->device);
  const int N = geom->n_bodies, M = bs[N];
  Work w;
  Arena sz{nullptr};
  carve(sz, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = ensure_ws(ctx, sz.off, s))) return rc;
  Arena ar{ctx->ws};
  carve(ar, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = setup(ctx, geom, bs, w, s))) return rc;
  if ((rc = fmm_setup(ctx->fmm, w.g, kind, &order, 1, s, ctx->err, fmm_schedule(M, kind, order).leaf_nodes)))
    return rc;
  const double* din;
  if ((rc = stage_in(ctx, in, w.io_in, (size_t)w.n, &din, s))) return rc;
  const bool dev_out = is_device_ptr(out);
  double* dout = dev_out ? out : w.io_out;
  const PairPlan one = uniform_plan(1, M);
  CK(fmm_pair_sum(ctx->fmm, w.g, kind, order, vec(const_cast<double*>(din)), w.g.w, w.partial, nullptr, s,
                  precision));
  CK(epilogue(w.g, kind, one, vec(const_cast<double*>(din)), w.partial, 0, 1, 1.0, vec(dout), nullptr, s));
  if (!dev_out) {
    CK(cudaMemcpyAsync(out, dout, (size_t)w.n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return BIE_OK;
}


size_t bie_workspace_bytes(int kind, int n_bodies, int n_nodes, int restart) {
  if (n_bodies < 1 || n_nodes < 1 || (kind != 0 && kind != 1)) return 0;
  // preconditioner blocks sized for bodies of equal size
  std::vector<int> bs(n_bodies + 1);
  for (int i = 0; i <= n_bodies; ++i) bs[i] = (int)((long long)n_nodes * i / n_bodies);
  return bie::workspace_bytes_for(kind, bs.data(), n_bodies, restart);
}

int bie_profile(bie_ctx* ctx, int enable, bie_profile_counters* out) {
  if (!ctx) return BIE_ERR_INVALID;
  DeviceGuard dg(ctx->device);
  resolve_timings(ctx, true);
  ctx->counters.kernel_launches = ctx->prof ? launches_so_far() - ctx->launch_mark : 0;
  if (out) *out = ctx->counters;
  if (enable) {
    memset(&ctx->counters, 0, sizeof(ctx->counters));
    ctx->launch_mark = launches_so_far();
  }
  ctx->prof = enable != 0;
  return BIE_OK;
}

void bie_destroy(bie_ctx* c) {
  if (!c) return;
  DeviceGuard dg(c->device);
  resolve_timings(c, true);
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (auto& gi : c->graphs) cudaGraphExecDestroy(gi.exec);
  if (c->fmm) bie::fmm_free(c->fmm, nullptr);
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
  }
  if (c->h_state) cudaFreeHost(c->h_state);
  if (c->h_small) cudaFreeHost(c->h_small);
  delete c;
}

const char* bie_last_error(const bie_ctx* c) { return c ? c->err.c_str() : "null context"; }

int elastance_solve(bie_ctx* ctx, const bie_geometry* geom, const double* q, double* phi, double* density,
                    const bie_opts* opts, bie_info* info, void* stream) {
  return solve_common(ctx, geom, 0, q, phi, density, opts, info, (cudaStream_t)stream);
}

int mobility_solve(bie_ctx* ctx, const bie_geometry* geom, const double* FT, double* UW, double* density,
                   const bie_opts* opts, bie_info* info, void* stream) {
  return solve_common(ctx, geom, 1, FT, UW, density, opts, info, (cudaStream_t)stream);
}

int elastance_solve_batch(bie_ctx* ctx, int count, const bie_geometry* geoms, const double* const* q,
                          double* const* phi, const bie_opts* opts, bie_info* info, int* status, void* stream) {
  const BatchIn b{count, geoms, q, phi, info, status};
  return solve_common(ctx, nullptr, 0, nullptr, nullptr, nullptr, opts, nullptr, (cudaStream_t)stream, &b);
}

int mobility_solve_batch(bie_ctx* ctx, int count, const bie_geometry* geoms, const double* const* FT,
                         double* const* UW, const bie_opts* opts, bie_info* info, int* status, void* stream) {
  const BatchIn b{count, geoms, FT, UW, info, status};
  return solve_common(ctx, nullptr, 1, nullptr, nullptr, nullptr, opts, nullptr, (cudaStream_t)stream, &b);
}

int bie_tune(bie_ctx* ctx, const bie_geometry* geom, int kind, int precision, int* splits, double* ms,
             void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> bs;
  int rc = validate(ctx, geom, bs);
  if (rc) return rc;
  if (kind != BIE_KIND_LAPLACE && kind != BIE_KIND_STOKES) return fail(ctx, BIE_ERR_INVALID, "bad kind");
  if (precision != BIE_PREC_FP64 && precision != BIE_PREC_MIXED && precision != BIE_PREC_MIXED_FF)
    return fail(ctx, BIE_ERR_INVALID, "bad precision");
  DeviceGuard dg(ctx->device);
  const int N = geom->n_bodies, M = bs[N];
  if (splits && *splits != 0) {  // install a plan, no timing
    if (*splits < 0 && (precision == BIE_PREC_FP64 || kind != BIE_KIND_LAPLACE))
      return fail(ctx, BIE_ERR_INVALID, "the symmetric plan exists for the FP32 and float-float Laplace pair sums only");
    const PairPlan p = *splits > 0 ? plan_with_splits(M, *splits) : plan_symmetric(M);
    set_tuned_plan(M, kind, precision, p);
    *splits = p.sym ? -p.S : p.S;
    if (ms) *ms = 0.0;
    return BIE_OK;
  }
  Work w;
  Arena sz{nullptr};
  carve(sz, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = ensure_ws(ctx, sz.off, s))) return rc;
  Arena ar{ctx->ws};
  carve(ar, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = setup(ctx, geom, bs, w, s))) return rc;
  // candidates: uniform split counts around the occupancy rule's, chunks of
  // whole source tiles (256 sources), and two-level plans (large chunks first,
  // small chunks last, so that the last wave drains fast)
  const PairPlan P0 = occupancy_plan(M, kind, precision);
  const int S0 = P0.S;
  std::vector<PairPlan> cand;
  auto add = [&](const PairPlan& p) {
    for (const PairPlan& q : cand)
      if (q.S == p.S && q.chunk == p.chunk && q.S1 == p.S1 && q.chunk2 == p.chunk2 && q.sym == p.sym) return;
    if (p.S >= 1 && p.chunk >= 1) cand.push_back(p);
  };
  add(P0);
  for (int c : {S0 / 2, (2 * S0) / 3, (3 * S0) / 2, 2 * S0, 3 * S0, 4 * S0, 6 * S0, 1}) add(plan_with_splits(M, std::max(1, c)));
  for (int t : {1, 2, 3, 4}) add(plan_with_splits(M, (M + 256 * t - 1) / (256 * t)));
  // the symmetric FP32 Laplace kernel, while its partials (one slot per tile) stay small
  if (precision != BIE_PREC_FP64 && kind == BIE_KIND_LAPLACE) {
    const PairPlan ps = plan_symmetric(M);
    if ((double)ps.S * M * sizeof(double) <= (1 << 30) && ps.S <= 4096) add(ps);
  }
  if (M >= 8192) {
    add(plan_two_level(M, 512, 128, 0.75));
    add(plan_two_level(M, 512, 256, 0.5));
    add(plan_two_level(M, 768, 256, 0.6));
    add(plan_two_level(M, 1024, 256, 0.75));
  }
  int smax = 1;
  for (const PairPlan& p : cand) smax = std::max(smax, p.S);
  // the timing scratch is released on every return path
  struct Scratch {
    double* partial = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s;
    ~Scratch() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (partial) cudaFreeAsync(partial, s);
    }
  } sc{nullptr, nullptr, nullptr, s};
  CK(cudaMallocAsync(reinterpret_cast<void**>(&sc.partial), (size_t)smax * w.n * sizeof(double), s));
  double* partial = sc.partial;
  CK(fill0(w.io_in, w.n, s));  // the cost of a pair sum does not depend on the values
  CK(cudaEventCreate(&sc.e0));
  CK(cudaEventCreate(&sc.e1));
  cudaEvent_t e0 = sc.e0, e1 = sc.e1;
  PairPlan best = P0;
  double best_ms = 0.0, s0_ms = 0.0;
  for (const PairPlan& p : cand) {
    auto apply = [&]() -> cudaError_t {
      cudaError_t e = pair_sum(w.g, kind, precision, p, vec(w.io_in), w.g.w, partial, nullptr, s);
      if (e != cudaSuccess) return e;
      return epilogue(w.g, kind, p, vec(w.io_in), partial, 0, 1, 1.0, vec(w.io_out), nullptr, s, 0.0,
                      precision == 1);
    };
    for (int it = 0; it < 2; ++it) CK(apply());
    // the fastest of five single applications
    double t_min = 1e300;
    for (int it = 0; it < 5; ++it) {
      CK(cudaEventRecord(e0, s));
      CK(apply());
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      t_min = std::min(t_min, (double)t);
    }
    if (&p == &cand[0]) s0_ms = t_min;
    if (best_ms == 0.0 || t_min < best_ms) {
      best_ms = t_min;
      best = p;
    }
  }
  CK(cudaStreamSynchronize(s));
  // keep the occupancy rule unless another plan is clearly faster (2%)
  if (best_ms > 0.98 * s0_ms) {
    best = P0;
    best_ms = s0_ms;
  }
  set_tuned_plan(M, kind, precision, best);
  if (splits) *splits = best.sym ? -best.S : best.S;
  if (ms) *ms = best_ms;
  return BIE_OK;
}

void bie_tune_clear(void) {
  clear_tuned_splits();
  std::lock_guard<std::mutex> lk(g_fmm_mu);
  g_fmm_sched.clear();
}

int bie_tune_fmm(bie_ctx* ctx, const bie_geometry* geom, int kind, const double* load, const bie_opts* opts,
                 int* leaf_nodes, int* inner_order, double* ms, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!ctx) return BIE_ERR_INVALID;
  if (kind != BIE_KIND_LAPLACE && kind != BIE_KIND_STOKES) return fail(ctx, BIE_ERR_INVALID, "bad kind");
  bie_opts o;
  fill_opts(opts, o);
  if (o.fmm_order < 2 || o.fmm_order > 64 || o.precision == BIE_PREC_FP64)
    return fail(ctx, BIE_ERR_INVALID, "bie_tune_fmm: a mixed precision and fmm_order in 2..64");
  std::vector<int> bs;
  int rc = validate(ctx, geom, bs);
  if (rc) return rc;
  if (!load) return fail(ctx, BIE_ERR_INVALID, "load is NULL");
  DeviceGuard dg(ctx->device);
  const int N = geom->n_bodies, M = bs[N], p = o.fmm_order;
  const int nout = kind == 0 ? N : 3 * N;
  struct Scratch {
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s;
    ~Scratch() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (out) cudaFreeAsync(out, s);
    }
  } sc{nullptr, nullptr, nullptr, s};
  CK(cudaMallocAsync(reinterpret_cast<void**>(&sc.out), nout * sizeof(double), s));
  CK(cudaEventCreate(&sc.e0));
  CK(cudaEventCreate(&sc.e1));
  // candidates: leaf populations around the default, and inner orders around
  // ceil(p/2) (a lower order is cheaper a matvec but may need more refinement
  // steps, so whole solves are timed); a candidate counts only if it converges
  const int pin0 = std::max(2, (p + 1) / 2);
  std::vector<FmmSchedule> cand;
  for (int leaf : {kDefaultLeafNodes, 12, 48})
    for (int pin : {pin0, pin0 - 4, pin0 - 2, pin0 + 2, pin0 + 4})
      if (pin >= 2 && pin <= p) cand.push_back(FmmSchedule{leaf, pin});
  const std::array<int, 4> key = fmm_key(M, kind, p);
  FmmSchedule best = cand[0];
  double best_ms = 0.0, def_ms = 0.0;
  bool any = false;
  for (size_t c = 0; c < cand.size(); ++c) {
    {
      std::lock_guard<std::mutex> lk(g_fmm_mu);
      g_fmm_sched[key] = cand[c];
    }
    double t_min = 1e300;
    bool ok = true;
    for (int it = 0; it < 3 && ok; ++it) {  // one warm-up, the faster of two
      CK(cudaEventRecord(sc.e0, s));
      bie_info info;
      const int st = solve_common(ctx, geom, kind, load, sc.out, nullptr, &o, &info, s);
      CK(cudaEventRecord(sc.e1, s));
      CK(cudaEventSynchronize(sc.e1));
      if (st < 0) {
        std::lock_guard<std::mutex> lk(g_fmm_mu);
        g_fmm_sched.erase(key);
        return st;
      }
      if (st == BIE_WARN_NOT_CONVERGED) ok = false;
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, sc.e0, sc.e1));
      if (it > 0) t_min = std::min(t_min, (double)t);
    }
    if (!ok) continue;
    if (c == 0) def_ms = t_min;
    if (!any || t_min < best_ms) {
      any = true;
      best_ms = t_min;
      best = cand[c];
    }
  }
  // keep the defaults unless another schedule is clearly faster (2%)
  if (def_ms > 0.0 && best_ms > 0.98 * def_ms) {
    best = cand[0];
    best_ms = def_ms;
  }
  {
    std::lock_guard<std::mutex> lk(g_fmm_mu);
    g_fmm_sched[key] = best;
  }
  if (leaf_nodes) *leaf_nodes = best.leaf_nodes;
  if (inner_order) *inner_order = best.inner_order;
  if (ms) *ms = best_ms;
  return BIE_OK;
}

void bie_test_arm_barrier_timeout(int skip_cta, long long spins) { arm_barrier_fault(skip_cta, spins); }

void bie_small_batch_path(int enable) { set_small_batch_path(enable != 0); }

void bie_test_precond_pivot_floor(double floor) { set_bj_pivot_floor(floor); }

int apply_operator(bie_ctx* ctx, const bie_geometry* geom, int kind, int precision, const double* in,
                   double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> bs;
  int rc = validate(ctx, geom, bs);
  if (rc) return rc;
  if (kind != BIE_KIND_LAPLACE && kind != BIE_KIND_STOKES) return fail(ctx, BIE_ERR_INVALID, "bad kind");
  if (precision != BIE_PREC_FP64 && precision != BIE_PREC_MIXED && precision != BIE_PREC_MIXED_FF)
    return fail(ctx, BIE_ERR_INVALID, "bad precision");
  if (!in || !out) return fail(ctx, BIE_ERR_INVALID, "in or out is NULL");
  if ((rc = check_local(ctx, {in, out}, "in or out"))) return rc;
  DeviceGuard dg(ctx->device);
  const int N = geom->n_bodies, M = bs[N];
  Work w;
  Arena sz{nullptr};
  carve(sz, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = ensure_ws(ctx, sz.off, s))) return rc;
  Arena ar{ctx->ws};
  carve(ar, w, N, M, kind, 1, false, true, geom->interior_pt != nullptr, false, true);
  if ((rc = setup(ctx, geom, bs, w, s))) return rc;
  const double* din;
  if ((rc = stage_in(ctx, in, w.io_in, (size_t)w.n, &din, s))) return rc;
  const PairPlan& p = precision == 0 ? w.plan64 : (precision == 1 ? w.plan32 : w.planff);
  const bool dev_out = is_device_ptr(out);
  double* dout = dev_out ? out : w.io_out;
  CK(timed_pair_sum(ctx, w.g, kind, precision, p, vec(const_cast<double*>(din)), w.g.w, w.partial, nullptr,
                    true, s));
  CK(epilogue(w.g, kind, p, vec(const_cast<double*>(din)), w.partial, 0, 1, 1.0, vec(dout), nullptr, s, 0.0,
              precision == 1));
  if (!dev_out) {
    CK(cudaMemcpyAsync(out, dout, (size_t)w.n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  return BIE_OK;
}

}  // extern "C"
