// Internal declarations shared by the translation units of libbie2d.
//
// Data layout in device memory (one staged geometry per call):
//   per node  [M]: x, y, nx, ny, w, sw = sqrt(w), kappa (float64),
//                  pf = (x_hi, y_hi, x_lo, y_lo) float4 with x = x_hi + x_lo exactly
//                  to ~2^-48 relative, nf = (nx, ny) float2, wkf = (sqrt(w), w kappa)
//                  float2, body_of (int32)
//   per body  [N]: len = |Gamma_i|, xc, yc (arc-length centroid), W_i, interior
//                  point z0 and stencil step delta, FP32 bounding box
//   densities: scaled by sqrt(w) (the L2 rescaling of Section 6.1.1); Stokes
//              vectors node-interleaved (2a + c).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bie2d.h"

namespace bie {

constexpr double kPi = 3.14159265358979323846;
constexpr double kInv2Pi = 0.15915494309189533577;  // 1/(2 pi)
constexpr double kInvPi = 0.31830988618379067154;   // 1/pi
constexpr double kInv4Pi = 0.07957747154594766788;  // 1/(4 pi)

// Batched GMRES (many independent problems in one block-diagonal system): each
// problem has its own Krylov space, Hessenberg matrix, rotations and stopping
// test; the problems advance in lockstep and a problem that has converged
// stops taking part.
struct PState {
  double tol_abs;  // stop threshold on this problem's residual estimate
  double beta;     // norm of the problem's starting residual in this cycle
  double res;      // residual estimate |g_{j+1}|
  double rnorm;    // last computed true residual norm
  double bnorm;    // norm of the problem's right-hand side
  int stop_j;      // steps of this cycle it took part in (INT_MAX: still active)
  int pad;
};
struct Geo {
  int N = 0, M = 0;
  const int* body_start = nullptr;  // [N+1]
  int* body_of = nullptr;           // [M]
  double *x = nullptr, *y = nullptr, *nx = nullptr, *ny = nullptr;
  double *w = nullptr, *sw = nullptr, *kappa = nullptr;
  float4* pf = nullptr;
  float2* nf = nullptr;
  float2* wkf = nullptr;  // [M] (sqrt(w), w kappa) in FP32, for the FP32 operator's epilogue
  double *len = nullptr, *xc = nullptr, *yc = nullptr, *W = nullptr;
  double *zx = nullptr, *zy = nullptr, *delta = nullptr, *wind = nullptr;
  float4* bbox = nullptr;  // [N] (xmin, ymin, xmax, ymax) of the body's nodes, FP32
  double* qscale = nullptr;  // [2] 2^Q and 2^(Q+23): quanta of the exact 3-float split of positions
  // exact 3-float split x = h + m + l of the positions (quanta from qscale) and
  // 2-float split of the normals, for the float-float pair sums
  float4* xff = nullptr;  // [M] (xh, xm, yh, ym)
  float2* xfl = nullptr;  // [M] (xl, yl)
  float4* nff = nullptr;  // [M] (nx_h, nx_l, ny_h, ny_l)
  // batched solves: [N] node range [x, y) of the problem each body belongs to
  // (pair and output sums stay inside a problem); nullptr: one problem [0, M)
  const int2* prange = nullptr;
  const int* pbody = nullptr;  // [nprob+1] first body of each problem (batched solves)
  int nprob = 1;
  // batched GMRES iterations only: a target block whose problems have all
  // stopped (stop_j <= *jstep) skips its pair sums and writes zero partials
  const PState* ps = nullptr;
  const int* bprob = nullptr;  // [N] problem of each body
  const int* jstep = nullptr;
  double pairs = 0.0;  // pair interactions of one operator application (0: M (M - 1))
  double* pnet = nullptr;  // [2 nprob] batched solves: each problem's net load and largest |load|
  float* qf = nullptr;     // [2M] scratch: FP32 source strengths of the FP32 pair sum
};

// A vector that lives at base + (idx ? *idx + off : off) * ld, so that a
// kernel can address the current Krylov vector without a host round trip.
struct VecRef {
  double* base;
  long long ld;
  const int* idx;
  int off;
  __device__ __forceinline__ double* ptr() const {
    return base + (long long)((idx ? *idx : 0) + off) * ld;
  }
};

inline VecRef vec(double* p) { return VecRef{p, 0, nullptr, 0}; }

// Device-side solver state (one per Krylov run).
struct KState {
  double tol_abs;  // stop threshold on the residual estimate
  double beta;     // norm of the cycle's starting residual
  double res;      // current residual estimate |g_{j+1}|
  double hnext;    // ||w|| after orthogonalisation (H[j+1][j] before rotation)
  double rnorm;    // last computed true residual norm
  double scratch[4];  // [0] relative tolerance, [1] norm of the right-hand side
  int j;           // iterations done in the current cycle
  int stop;        // 1 when the cycle has ended (converged, full or breakdown)
  int iters;       // iterations over all cycles
  int maxit;       // iteration cap over all cycles
  int m;           // restart length
  int counter;     // last-block-done counter for grid reductions
  int pad[2];         // [0] = 1: set tol_abs from the next starting residual
  unsigned bar_count, bar_gen;  // grid barrier of the fused Arnoldi step
  int error;          // 1: a grid barrier gave up waiting (results invalid)
  int nactive;        // batched GMRES: problems still iterating in this cycle
};

struct SegArgs {
  int P = 0;                      // problems (0: one system, not segmented)
  int nitem = 0;                  // element ranges of the fused Arnoldi step
  const long long* pnode = nullptr;  // [P+1] first vector entry of each problem
  const long long* ibeg = nullptr;   // [nitem+1] ranges, none crossing a problem
  const int* iprob = nullptr;        // [nitem] problem of each range
  const int* pitem = nullptr;        // [P+1] first range of each problem
  const int* bprob = nullptr;        // [N] problem of each body
  PState* ps = nullptr;              // [P]
};

}  // namespace bie
struct bie_ctx;
namespace bie {
// Return a context's workspace to the stream-ordered pool (used by the server
// between requests, so that memory follows the requests in flight).
void release_workspace(bie_ctx* ctx, cudaStream_t s);

// Count of kernels launched by this library (all contexts), for bie_profile.
void note_launches(int k);
long long launches_so_far();

// ---------------------------------------------------------------- geometry.cu
// Stage the geometry: weights, normals, curvature, per-body length/centroid/W,
// interior points, winding numbers, FP32 hi/lo coordinates.
cudaError_t stage_geometry(const Geo& g, const double* x, const double* y, const double* dx,
                           const double* dy, const double* ddx, const double* ddy,
                           const double* interior_pt, cudaStream_t s);

// f (scaled) for the total-density formulation: sw_a * q_i (Laplace) or
// sw_a * (F_i + T_i p_a) (Stokes).
cudaError_t total_density_rhs(const Geo& g, int kind, const double* load, double* f, cudaStream_t s);
// Incident density scaled by sw: sw*sigma (Laplace) or sw*rho (Stokes).
cudaError_t incident_density_scaled(const Geo& g, int kind, const double* load, double* out,
                                    cudaStream_t s);

// Output evaluation at interior points from v = sw * nu (scaled total density).
// Laplace: out[i] = phi_i; Stokes: out[3i..3i+2] = (vx, vy, omega).  Also writes
// the constraint residual max over bodies into *cres (device) relative to the load.
cudaError_t evaluate_output(const Geo& g, int kind, const double* v, const double* load,
                            double* partial, int P, double* out, double* cres, cudaStream_t s);
int output_splits(const Geo& g, int kind);
// the second half of evaluate_output, on sums already in partial (P splits)
cudaError_t finalize_output(const Geo& g, int kind, const double* v, const double* load, double* partial, int P,
                            double* out, double* cres, cudaStream_t s);

// elementwise helpers
cudaError_t unscale(const Geo& g, int kind, const double* v, double* out, cudaStream_t s);   // v/sw
cudaError_t scale_by(const Geo& g, int kind, const double* in, const double* fac, double* out,
                     cudaStream_t s);  // out = fac*in (fac per node)
cudaError_t net_load(int N, int kind, const double* load, double* out, cudaStream_t s);

// ---------------------------------------------------------------- pairsum.cu
// Streaming multiprocessors of the current device (queried once per device).
int device_sms();

// partial[s][a] (scalar for Laplace, 2-vector for Stokes) = sum over sources b
// of split s, b != a, of the kernel without its constant, with source strength
// sscale_b * v_b.  FP64 and FP32 variants.
// Source splits of a pair sum: splits s < S1 take `chunk` sources each, the
// remaining S - S1 splits `chunk2` each (a two-level plan: large chunks are
// dispatched first and small ones last, so that the last wave drains fast).
// Uniform plans have S1 = S.  Batched solves use `chunk` only.
struct PairPlan {
  int S;         // source splits
  int chunk;     // sources per split (the first S1 splits)
  int S1;        // splits of `chunk` sources
  int chunk2;    // sources per split after the first S1
  int sym = 0;   // FP32 Laplace: the symmetric kernel (S = tiles of 256 nodes, one CTA per tile pair)
};
inline PairPlan uniform_plan(int S, int chunk) { return PairPlan{S, chunk, S, chunk}; }
// the tuned split count of this shape (bie_tune) if any, else occupancy_plan:
// one wave of blocks (target blocks x splits) over every SM
PairPlan plan_pairs(int M, int kind, int precision);
PairPlan occupancy_plan(int M, int kind, int precision);
PairPlan plan_with_splits(int M, int S);
// two-level plan: a fraction f of the sources in chunks of c1, the rest in chunks of c2
PairPlan plan_two_level(int M, int c1, int c2, double f);
// the symmetric FP32 Laplace pair sum (partials: one slot per 256-node tile)
PairPlan plan_symmetric(int M);
void set_tuned_plan(int M, int kind, int precision, const PairPlan& p);
void forget_tuned_plan(int M, int kind, int precision);
void clear_tuned_splits();
// batched solves (host arrays: body_start [N+1], first body of each problem [P+1])
PairPlan plan_pairs_batch(const int* body_start, int N, const int* pbody, int P, int kind, int precision);
cudaError_t pair_sum(const Geo& g, int kind, int precision, const PairPlan& p, VecRef v,
                     const double* sscale, double* partial, const int* stop, cudaStream_t s);

// out = sign * [ 1/2 v + oscale * (K v + diag + [L] v) ] with the constants applied.
// scaled = 1: v is sqrt(w)-scaled, source strength sw, output scaled by sw.
// scaled = 0: v unscaled, source strength w, output unscaled.
// alpha = 0: the paper's completion L; alpha > 0: L weighted per body by
// alpha/|Gamma_i| (force part) and alpha/W_i (torque part).
// pff: the partials are float-float pairs (written by the FP32 pair sums,
// precision 1), summed in float-float; otherwise doubles.
cudaError_t epilogue(const Geo& g, int kind, const PairPlan& p, VecRef v, const double* partial,
                     int scaled, int with_L, double sign, VecRef out, const int* stop,
                     cudaStream_t s, double alpha = 0.0, bool pff = false, bool fp32 = false);
// out = in - (I - C) L~(in) for a correction solved with the weighted completion.
cudaError_t consistent_rhs(const Geo& g, int kind, double alpha, const double* in, double* out,
                           cudaStream_t s);

// ---------------------------------------------------------------- fmm.cu
struct FmmState;
// Build the quadtree for the staged geometry and the translation operators of
// every order in `orders` (at most 64).  One host round trip.
// leaf_nodes: the leaf level is the finest whose non-empty leaves hold at
// least that many nodes (<= 0: kDefaultLeafNodes).
constexpr int kDefaultLeafNodes = 24;
int fmm_setup(FmmState*& f, const Geo& g, int kind, const int* orders, int norders, cudaStream_t s,
              std::string& err, int leaf_nodes = 0);
// FMM schedule of a shape (device, M, kind, residual order): leaf population
// and the order of the inner solves' FMM, as tuned by bie_tune_fmm (else the
// defaults: kDefaultLeafNodes and ceil(order / 2)).
struct FmmSchedule {
  int leaf_nodes;
  int inner_order;
};
FmmSchedule fmm_schedule(int M, int kind, int order);
// Pair sums by the FMM of order p into partial (layout of a single source
// split); the near field in FP64 (near_prec 0), FP32 (1) or float-float (2).
cudaError_t fmm_pair_sum(FmmState* f, const Geo& g, int kind, int p, VecRef v, const double* sscale,
                         double* partial, const int* stop, cudaStream_t s, int near_prec = 0);
void fmm_free(FmmState* f, cudaStream_t s);
// Output single layers at the interior targets by the FMM (one split, the
// layout of evaluate_output's direct sums).
// What a captured FMM application depends on besides its arguments: the
// tree's buffers, level count and bounding square (baked into the captured
// launches); two values that change whenever any of them does.
void fmm_signature(const FmmState* f, long long sig[2]);
cudaError_t fmm_output(FmmState* f, const Geo& g, int kind, int p, const double* v, double* part, cudaStream_t s,
                       bool ff = false);

// workspace of a solve with the given host body_start (bie_workspace_bytes assumes equal bodies)
size_t workspace_bytes_for(int kind, const int* body_start_host, int n_bodies, int restart);
// workspace of a batched solve (host arrays: concatenated body_start [N+1],
// first body of each problem [nprob+1])
size_t workspace_bytes_batch(int kind, const int* bs, int n_bodies, const int* pb, int nprob, const bie_opts* opts);

// Batched solves: per-problem unit-norm scaling of f (pnode = entry offsets
// of the problems) and the inverse scaling of the solution.
cudaError_t batch_normalize(int nprob, const long long* pnode, double* f, double* scale, cudaStream_t s);
cudaError_t batch_unscale(int nprob, const long long* pnode, const double* scale, double* x, cudaStream_t s);
// Many small device-to-device copies in one launch (batched solves): segment
// i copies words 4-byte words from src to dst; the table is uploaded to a
// stream-ordered temporary buffer.
struct CopySeg {
  const void* src;
  void* dst;
  long long words;
};
cudaError_t gather_segments(const std::vector<CopySeg>& segs, cudaStream_t s);
// norms[p] = ||x_p|| per problem; x_p = 0 where norms[p] <= thr
cudaError_t seg_norms(int nprob, const long long* pnode, const double* x, double* norms, cudaStream_t s);
cudaError_t seg_zero_below(int nprob, const long long* pnode, const double* norms, double thr, double* x,
                           cudaStream_t s);

// ---------------------------------------------------------------- precond.cu
// Largest per-body block (unknowns) that the block-Jacobi preconditioner inverts.
constexpr int kBjMaxBlock = 640;

// Block-Jacobi (per body) preconditioner: each body's diagonal block of the
// operator GMRES iterates on (alpha = 0: the paper's completion; alpha > 0:
// the completion weighted by alpha/|Gamma_i|, alpha/W_i), inverted in FP32.  A
// block whose inversion meets a pivot that is not finite or below the floor
// (|p| < floor; the blocks are 1/2 I + compact) keeps the identity, and
// *fallbacks (device int, cleared here) counts those bodies.
// Storage: per body W = B^{-1} - 2I (B^{-1} = 2I + O(compact)) in FP16,
// column-major; P v = 2 v + W v.  An inverse with an entry of W outside
// FP16's range also keeps the identity (W = -I).
using bj_t = __half;
constexpr float kBjShift = 2.0f;
long long bj_block_floats(const int* body_start_host, int N, int kind);
cudaError_t bj_setup(const Geo& g, int kind, double alpha, const int* body_start_host, long long* off_dev,
                     int* pair_dev, bj_t* blocks, int* fallbacks, cudaStream_t s);
// Test hook: the pivot floor of later factorisations (<= 0: the default).
void set_bj_pivot_floor(double floor);
// z = P v (v scaled, z scaled); f64: in FP64 arithmetic on the FP16 blocks
cudaError_t bj_apply(const Geo& g, int kind, const long long* off_dev, const bj_t* blocks, VecRef v, double* z,
                     const int* stop, int max_nb, cudaStream_t s, bool f64 = false);

// ---------------------------------------------------------------- small.cu
// One-launch solves of batches of small problems (one CTA per problem, the
// whole float-float refinement inside it).
constexpr int kSmallMaxNodes = 1024;
constexpr int kSmallMaxBodies = 128;
struct SmallInfo {
  int iters, refinements, matvecs32, matvecsff;
  double rel_residual, fp32_error;
};
bool small_batch_eligible(int max_nodes, int max_bodies, int restart);
// Every problem p of the batch: solve the sqrt(w)-scaled total-density system
// with right-hand side f (batch layout, per-problem entries [pnode[p],
// pnode[p+1]), bodies [pbody[p], pbody[p+1])) into x, to tol relative to its
// own ||f||; r, d, rc, rin, y are batch-layout scratch vectors and V the basis
// rows (V + i ld).  info[p] receives the counts.
cudaError_t small_batch_solve(const Geo& g, int kind, int P, const int* pbody, const long long* pnode,
                              const double* f, double* x, double* r, double* d, double* rc, double* rin, double* y,
                              double* V, long long ld, int m, double tol, double inner_tol, int max_refine,
                              int max_iter, int max_nodes, SmallInfo* info, cudaStream_t s);
// the one-launch path for batches of small problems: on (default) or off
void set_small_batch_path(bool on);
bool small_batch_path();

// ---------------------------------------------------------------- krylov.cu
constexpr int kMaxVecGrid = 608;  // largest grid of the vector kernels and the Arnoldi step
int vec_grid(long long n);

// One fused Arnoldi step (CGS2, norm, Givens, normalisation and optionally
// z = P v_{j+1}); part holds [3][grid][201] doubles.
struct ArnoldiArgs {
  double* V;
  long long ld, n;
  KState* st;
  double *part, *H, *cs, *sn, *gv;
  // block-Jacobi preconditioner: blocks == nullptr for none
  Geo g;
  int kind;
  const long long* off;
  const bj_t* blocks;
  double* z;
  int bj64 = 0;            // apply the FP32 blocks in FP64 arithmetic (FP64 GMRES)
  float* vf = nullptr;     // FP32 copy of the basis ((m + 1) x ld): CGS2 in FP32 (FP32 inner solves, wide grids)
  int fault_skip = -1;     // test hook: this CTA leaves before the first grid barrier
  long long spins = 0;     // polls before a grid barrier gives up (set by the launcher)
};
// Test hook of the bounded barrier waits: the next Arnoldi launch skips CTA
// skip_cta and gives up waiting after `spins` polls (spins <= 0: disarmed).
void arm_barrier_fault(int skip_cta, long long spins);
bool barrier_fault_armed();
// co-resident CTAs for the cooperative launch (fp32: the FP32 step of wide grids)
int arnoldi_grid(long long n, bool fp32 = false, int nbodies = 0);
bool arnoldi_narrow(long long n);
cudaError_t arnoldi(const ArnoldiArgs& a, int grid, cudaStream_t s);
// h[i] = <V_i, w> for i <= j (first CGS pass)

// Batched GMRES: the same Arnoldi step per problem (H, cs, sn, gv hold P
// consecutive copies: [P][m][m+1], [P][m], [P][m], [P][m+1]); part holds
// [3][nitem][201] doubles.
int arnoldi_seg_grid(long long n);
cudaError_t arnoldi_seg(const ArnoldiArgs& a, const SegArgs& sg, int grid, cudaStream_t s);
// per problem p: r = f - y over its entries, rnorm_p; opens a cycle: V0 = r/rnorm_p
// (zero for a problem already below its tolerance), g_p = (rnorm_p, 0, ..)
cudaError_t residual_start_seg(const double* f, const double* y, double* r, double* V0, KState* st,
                               const SegArgs& sg, double* gv, int m, cudaStream_t s);
// per problem: y_p = R_p^{-1} g_p over the steps it took part in, x += V y_p
cudaError_t gmres_update_seg(const double* V, long long ld, KState* st, const SegArgs& sg, const double* H,
                             const double* gv, double* y, double* x, int m, long long max_len, cudaStream_t s);

// y = R^{-1} g and x += V y
cudaError_t gmres_update(const double* V, long long ld, long long n, KState* st, const double* H,
                         const double* gv, double* y, double* x, int grid, cudaStream_t s);
// r = f - y, rnorm = ||r||; also optionally starts a cycle: V0 = r/rnorm, g = (rnorm, 0..)
cudaError_t residual_start(const double* f, const double* y, double* r, double* V0, long long n,
                           KState* st, double* part, double* gv, int start_cycle, int grid,
                           cudaStream_t s);
cudaError_t axpy(double* x, const double* d, long long n, cudaStream_t s);  // x += d
cudaError_t fill0(double* x, long long n, cudaStream_t s);

}  // namespace bie
