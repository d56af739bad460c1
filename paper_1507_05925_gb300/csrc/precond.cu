// Block-Jacobi preconditioner of the GMRES iterations: the FP32 inner solves
// of the refinement (operator with the per-body weighted completion) and the
// FP64 GMRES (the paper's completion).
//
// The operator is the second-kind operator, sqrt(w)-scaled.  Its diagonal
// block for body i,
//   B_i = 1/2 I + D (K_ii + C_i L_ii) D^{-1}     (Laplace: n_i x n_i; Stokes: 2n_i x 2n_i)
// (C_i = 1 for the paper's L) is assembled in FP32 (from hi/lo coordinate
// differences) directly in shared memory and inverted in place by blocked
// Gauss-Jordan elimination without pivoting: the blocks are 1/2 I + compact,
// their pivots stay near 1/2 on the shapes measured (0.36 - 0.50) and an FP32
// inverse accurate to ~1e-6 is far more than a preconditioner needs.  Every
// pivot is checked: one that is not finite or smaller in magnitude than the
// floor (default 1e-3, 1/500 of the identity part), or a non-finite entry of
// the finished inverse, makes the body keep the identity block (counted in
// bie_info.precond_fallbacks), so a nearly singular block can slow GMRES down
// but never poisons it with NaN or huge entries.  A block of
// nb <= 128 unknowns is inverted by one CTA; nb <= 448 by a cluster of four
// CTAs and nb <= 640 by one of eight, each CTA holding a slice of the columns
// and reading the pivot panels of the others through distributed shared
// memory; larger blocks are left as the identity.  The inverses are stored
// column-major as W = B^{-1} - 2I in FP16 (half the bytes of the apply, which
// streams every block once a GMRES iteration: 655 MB in FP32 for 10,000
// bodies of 128 unknowns).  B^{-1} is 2I plus a compact part, so W carries
// FP16's 2^-11 relative precision on that part only; a perturbed
// preconditioner is still one fixed linear map and changes iteration counts
// at most.  P v = 2 v + W v.  Preconditioning is applied from the right,
// z = P v, so the GMRES residual stays the true residual.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"
#include "reduce.cuh"

namespace cg = cooperative_groups;

namespace bie {

namespace {

constexpr int kMaxSingle = 128;  // one CTA
constexpr int kMaxBlock4 = 448;  // cluster of four CTAs
constexpr int kMaxBlock = kBjMaxBlock;  // cluster of eight CTAs (640); larger bodies keep the identity
constexpr int kPB = 16;          // panel width of the blocked elimination
constexpr int kMaxThreads = 640; // one thread per row
constexpr int kBA = 256;         // threads of an application CTA
constexpr int kApplyRows = 64, kApplyGroups = kBA / kApplyRows;

// Shared-memory leading dimension of a column: odd, so that reading a row
// (stride ld across threads) is free of bank conflicts.
__host__ __device__ __forceinline__ int gj_ld(int nb) { return nb | 1; }
// Columns per CTA of a cluster of cs CTAs: a multiple of the panel width, so
// that each panel lies in one CTA.
__host__ __device__ __forceinline__ int gj_cols(int nb, int cs) {
  return ((nb + cs - 1) / cs + kPB - 1) / kPB * kPB;
}
__host__ __device__ __forceinline__ size_t gj_smem_floats(int nb, int cs) {
  const int h = gj_cols(nb, cs);
  return (size_t)gj_ld(nb) * h + (size_t)h * kPB + 2 * kPB + 8 * (size_t)h;
}

// Entry (row r, column c) of the operator's diagonal block of body i
// (sqrt(w)-scaled; alpha > 0: completion weighted by alpha/|Gamma_i| and
// alpha/W_i, alpha = 0: the paper's completion), in FP32: coordinate differences from
// the hi/lo split (x = x_hi + x_lo, exact leading differences as in the near
// tiles of the pair sum), the column's node data staged in shared memory.
struct BlockRow {
  int kind, a;
  float cf, ct;
  float4 pa;  // (x_hi, y_hi, x_lo, y_lo) of the row's node
  float nxa, nya, swa, ka, pa0, pa1;
  int al;
  __device__ BlockRow(const Geo& g, int kind_, int i, int r, double alpha) : kind(kind_) {
    const int a0 = g.body_start[i];
    cf = alpha > 0.0 ? (float)(alpha / g.len[i]) : 1.0f;
    ct = kind == 1 ? (alpha > 0.0 ? (float)(alpha / g.W[i]) : 1.0f) : 0.f;
    a = a0 + (kind == 1 ? r >> 1 : r);
    al = kind == 1 ? r & 1 : 0;
    pa = g.pf[a];
    const float2 n = g.nf[a];
    nxa = n.x;
    nya = n.y;
    swa = (float)g.sw[a];
    ka = (float)g.kappa[a];
    pa0 = (float)(-(g.y[a] - g.yc[i]));
    pa1 = (float)(g.x[a] - g.xc[i]);
  }
  // column data: cp = (x_hi, y_hi, x_lo, y_lo), cw = (sqrt(w), p_1, p_2, node index)
  __device__ float entry(int r, int c, float4 cp, float4 cw) const {
    const int b = __float_as_int(cw.w);
    const float swb = cw.x;
    const float rx = (pa.x - cp.x) + (pa.z - cp.z), ry = (pa.y - cp.y) + (pa.w - cp.w);
    float k;
    if (kind == 0) {
      if (a == b) {
        k = -ka * (float)kInv4Pi;
      } else {
        k = -(float)kInv2Pi * (rx * nxa + ry * nya) / (rx * rx + ry * ry);
      }
      return (r == c ? 0.5f : 0.f) + swa * swb * (k + cf);
    }
    const int be = c & 1;
    if (a == b) {
      const float t = al == 0 ? -nya : nxa, u = be == 0 ? -nya : nxa;
      k = -0.5f * (float)kInvPi * ka * t * u;
    } else {
      const float r2 = rx * rx + ry * ry;
      const float rn = rx * nxa + ry * nya;
      k = -(float)kInvPi * (al == 0 ? rx : ry) * (be == 0 ? rx : ry) * rn / (r2 * r2);
    }
    const float pb = be == 0 ? cw.y : cw.z;
    const float pa_ = al == 0 ? pa0 : pa1;
    return (r == c ? 0.5f : 0.f) + swa * swb * (k + (al == be ? cf : 0.f) + ct * pa_ * pb);
  }
};

// A_:j += F G_j for the local columns [j0, j1) of row r (F = this row of the
// panel minus E_K, G_j = rows K of column j).
__device__ __forceinline__ void rank_update(float* __restrict__ A, const float* __restrict__ G, int h, int ld, int r,
                                            const float (&fr)[kPB], int j0, int j1) {
  // G is [kPB][h] (panel row t of the local columns): one 16-byte load gives
  // four columns of one row, added with packed FP32x2 multiply-adds; each
  // column's terms in the order t = 0, 1, ..., as one column at a time
  int j = j0;
  for (; j < j1 && (j & 3); ++j) {
    float acc = A[j * ld + r];
#pragma unroll
    for (int t = 0; t < kPB; ++t) acc = fmaf(fr[t], G[t * h + j], acc);
    A[j * ld + r] = acc;
  }
  for (; j + 4 <= j1; j += 4) {
    float2 a01 = make_float2(A[j * ld + r], A[(j + 1) * ld + r]);
    float2 a23 = make_float2(A[(j + 2) * ld + r], A[(j + 3) * ld + r]);
#pragma unroll
    for (int t = 0; t < kPB; ++t) {
      const float4 g = *reinterpret_cast<const float4*>(G + t * h + j);
      const float2 f = make_float2(fr[t], fr[t]);
      a01 = __ffma2_rn(f, make_float2(g.x, g.y), a01);
      a23 = __ffma2_rn(f, make_float2(g.z, g.w), a23);
    }
    A[j * ld + r] = a01.x;
    A[(j + 1) * ld + r] = a01.y;
    A[(j + 2) * ld + r] = a23.x;
    A[(j + 3) * ld + r] = a23.y;
  }
  for (; j < j1; ++j) {
    float acc = A[j * ld + r];
#pragma unroll
    for (int t = 0; t < kPB; ++t) acc = fmaf(fr[t], G[t * h + j], acc);
    A[j * ld + r] = acc;
  }
}

// Assembly and in-place inversion of one diagonal block by a cluster of CS CTAs
// (CS = 1: one CTA).  CTA q holds the columns [q h, min(nb, (q+1) h)) and all
// rows, one thread per row.  Blocked Gauss-Jordan without pivoting: for each
// panel K of kPB pivots, the owning CTA eliminates the panel's own columns in
// registers, after which its columns hold [inv(A_KK); -A_RK inv(A_KK)]; every
// CTA then applies the rank-kPB update A_:j += (panel - E_K) A_Kj to its other
// columns, reading the panel from the owner's shared memory.  The panel stays
// unchanged until the owner's next update, which follows the next panel's
// cluster barrier, which no CTA reaches before it is done reading.
// Launch bounds per cluster size: one thread per row of the largest block the
// instance takes; the clusters of four keep at least two CTAs of 448 threads
// (three of 256) on an SM.
template <int CS>
__global__ void __launch_bounds__(CS == 1 ? kMaxSingle : CS == 4 ? kMaxBlock4 : kMaxThreads, CS == 4 ? 2 : 1)
    k_bj_factor(Geo g, int kind, double alpha,
                                                           const int* __restrict__ list,
                                                           const long long* __restrict__ off,
                                                           bj_t* __restrict__ blocks, float floor,
                                                           int* __restrict__ fallbacks) {
  extern __shared__ float sm[];
  __shared__ int bad_s;  // this CTA met a bad pivot or a non-finite entry
  const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
  const int i = list[blockIdx.x / CS];
  const int nb = (g.body_start[i + 1] - g.body_start[i]) * (kind + 1);
  const int ld = gj_ld(nb), h = gj_cols(nb, CS);
  const int c0 = min(nb, rank * h), nc = min(nb, c0 + h) - c0;
  float* A = sm;                 // ld x h, column-major
  float* G = A + (size_t)ld * h; // kPB x h: rows K of the local columns
  float* rowbuf = G + (size_t)h * kPB;  // [2][kPB] pivot rows of the panel steps
  float4* colp = reinterpret_cast<float4*>(rowbuf + 2 * kPB);  // [h] column node positions
  float4* colw = colp + h;                                       // [h] column node data
  const int r = threadIdx.x;
  const bool live = r < nb;
  if (threadIdx.x == 0) bad_s = 0;
  {
    const int a0 = g.body_start[i];
    const double xc = g.xc[i], yc = g.yc[i];
    for (int j = threadIdx.x; j < nc; j += blockDim.x) {
      const int c = c0 + j;
      const int b = a0 + (kind == 1 ? c >> 1 : c);
      colp[j] = g.pf[b];
      colw[j] = make_float4((float)g.sw[b], (float)(-(g.y[b] - yc)), (float)(g.x[b] - xc), __int_as_float(b));
    }
  }
  __syncthreads();
  if (live) {
    const BlockRow br(g, kind, i, r, alpha);
    for (int j = 0; j < nc; ++j) A[j * ld + r] = br.entry(r, c0 + j, colp[j], colw[j]);
  }
  __syncthreads();
  for (int k0 = 0; k0 < nb; k0 += kPB) {
    const int bsz = min(kPB, nb - k0);
    const int owner = k0 / h;
    if (rank == owner) {
      // panel elimination in registers: thread r holds row r of the panel
      const int lj = k0 - c0;
      float pr[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) pr[t] = (live && t < bsz) ? A[(lj + t) * ld + r] : 0.f;
#pragma unroll
      for (int t = 0; t < kPB; ++t) {
        if (t < bsz) {
          float* rb = rowbuf + (t & 1) * kPB;
          if (r == k0 + t) {
#pragma unroll
            for (int u = 0; u < kPB; ++u) rb[u] = pr[u];
          }
          __syncthreads();
          const float pv = rb[t];
          if (threadIdx.x == 0 && !(fabsf(pv) >= floor && isfinite(pv))) bad_s = 1;
          const float ip = 1.0f / pv;
          if (r == k0 + t) {
#pragma unroll
            for (int u = 0; u < kPB; ++u) pr[u] = (u == t) ? ip : pr[u] * ip;
          } else {
            const float fr = pr[t] * ip;
#pragma unroll
            for (int u = 0; u < kPB; ++u) pr[u] = (u == t) ? -fr : fmaf(-fr, rb[u], pr[u]);
          }
        }
      }
      if (live) {
#pragma unroll
        for (int t = 0; t < kPB; ++t)
          if (t < bsz) A[(lj + t) * ld + r] = pr[t];
      }
    }
    // rows K of the local columns, before any of them changes
    for (int e = threadIdx.x; e < nc * bsz; e += blockDim.x) {
      const int j = e / bsz, t = e % bsz;
      G[t * h + j] = A[j * ld + k0 + t];
    }
    if constexpr (CS > 1) {
      cg::this_cluster().sync();
    } else {
      __syncthreads();
    }
    if (live) {
      const float* P = A + (k0 - owner * h) * ld;  // the panel in the owner's shared memory
      if constexpr (CS > 1) P = cg::this_cluster().map_shared_rank(P, owner);
      float fr[kPB];
#pragma unroll
      for (int t = 0; t < kPB; ++t) fr[t] = t < bsz ? P[t * ld + r] - (r == k0 + t ? 1.f : 0.f) : 0.f;
      // all local columns but the panel's own (owner: [k0 - c0, k0 - c0 + bsz))
      const int s0 = rank == owner ? k0 - c0 : nc, s1 = rank == owner ? k0 - c0 + bsz : nc;
      rank_update(A, G, h, ld, r, fr, 0, s0);
      rank_update(A, G, h, ld, r, fr, s1, nc);
    }
    __syncthreads();
  }
  // an entry that overflowed in the updates, or whose W = B^{-1} - 2I entry
  // lies outside FP16's range, also rejects the block
  if (live) {
    bool nf = false;
    for (int j = 0; j < nc; ++j) {
      const float a = A[j * ld + r] - (c0 + j == r ? kBjShift : 0.f);
      nf |= !(fabsf(a) <= 65000.f);
    }
    if (nf) bad_s = 1;
  }
  // every CTA of the cluster learns whether any of them rejected the block
  // (the first sync also keeps every CTA alive while the last panel is read)
  int bad;
  if constexpr (CS > 1) {
    cg::this_cluster().sync();
    bad = 0;
    for (int q = 0; q < CS; ++q) bad |= *cg::this_cluster().map_shared_rank(&bad_s, q);
    cg::this_cluster().sync();
  } else {
    __syncthreads();
    bad = bad_s;
  }
  if (bad && rank == 0 && threadIdx.x == 0) atomicAdd(fallbacks, 1);
  bj_t* B = blocks + off[i];
  if (live)
    for (int j = 0; j < nc; ++j) {
      const float d = c0 + j == r ? kBjShift : 0.f;  // W = B^{-1} - 2I; the identity: W = -I
      B[(long long)(c0 + j) * nb + r] = __float2half_rn(bad ? (c0 + j == r ? 1.f : 0.f) - d : A[j * ld + r] - d);
    }
}

// z = P v: z_i = B_i^{-1} v_i per body (identity for bodies left out).  CTA
// (i, y) computes rows [64 y, 64 y + 64) of body i with four column groups of
// 64 threads, reduced in shared memory; each warp reads 32 consecutive rows of
// one column (coalesced).
// F64: the same product in FP64 arithmetic (v not rounded to FP32), so that
// P is one fixed linear map to FP64 rounding (FP64 GMRES).
template <bool F64>
__global__ void __launch_bounds__(kBA) k_bj_apply(Geo g, int kind, const long long* __restrict__ off,
                                                  const bj_t* __restrict__ blocks, VecRef vr, double* __restrict__ z,
                                                  const int* __restrict__ stop) {
  using T = typename std::conditional<F64, double, float>::type;
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char vs_raw[];
  T* vs = reinterpret_cast<T*>(vs_raw);
  __shared__ T part[kBA];
  const double* v = vr.ptr();
  const int i = blockIdx.x;
  const int c = kind + 1;
  const int a0 = g.body_start[i] * c, nb = (g.body_start[i + 1] - g.body_start[i]) * c;
  const int r0 = blockIdx.y * kApplyRows;
  if (r0 >= nb) return;
  const int lr = threadIdx.x % kApplyRows, grp = threadIdx.x / kApplyRows;
  const int r = r0 + lr;
  if (nb > kMaxBlock) {
    if (grp == 0 && r < nb) z[a0 + r] = v[a0 + r];
    return;
  }
  for (int e = threadIdx.x; e < nb; e += kBA) vs[e] = (T)v[a0 + e];
  __syncthreads();
  const bj_t* B = blocks + off[i];
  T acc = 0;
  if (r < nb) {
    const int per = (nb + kApplyGroups - 1) / kApplyGroups;
    const int cb = grp * per, ce = min(nb, cb + per);
#pragma unroll 4
    for (int col = cb; col < ce; ++col) acc = fma((T)__half2float(B[(long long)col * nb + r]), vs[col], acc);
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (grp == 0 && r < nb) {
    T t = part[lr];
#pragma unroll
    for (int q = 1; q < kApplyGroups; ++q) t += part[q * kApplyRows + lr];
    z[a0 + r] = (double)(fma((T)kBjShift, vs[r], t));  // P v = 2 v + W v
  }
}

}  // namespace

long long bj_block_floats(const int* body_start_host, int N, int kind) {
  long long s = 0;
  for (int i = 0; i < N; ++i) {
    const long long nb = (long long)(body_start_host[i + 1] - body_start_host[i]) * (kind + 1);
    if (nb <= kMaxBlock) s += nb * nb;
  }
  return s;
}

namespace {

// Launch of k_bj_factor<CS> over count bodies of list, one thread per row.
float g_pivot_floor = 0.f;  // test hook (0: the default floor)
constexpr float kPivotFloor = 1e-3f;

template <int CS>
cudaError_t launch_factor(const Geo& g, int kind, double alpha, const int* list, int count, int threads, size_t smem,
                          const long long* off, bj_t* blocks, int* fallbacks, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_bj_factor<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CS * count);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = CS > 1 ? 1 : 0;
  const float floor = g_pivot_floor > 0.f ? g_pivot_floor : kPivotFloor;
  e = cudaLaunchKernelEx(&cfg, k_bj_factor<CS>, g, kind, alpha, list, off, blocks, floor, fallbacks);
  note_launches(1);
  return e;
}

}  // namespace

void set_bj_pivot_floor(double floor) { g_pivot_floor = floor > 0.0 ? (float)floor : 0.f; }

cudaError_t bj_setup(const Geo& g, int kind, double alpha, const int* body_start_host, long long* off_dev,
                     int* list_dev, bj_t* blocks, int* fallbacks, cudaStream_t s) {
  // bodies by kernel: one CTA (nb <= 128), clusters of four (<= 448) and eight (<= 640) CTAs
  constexpr int kCs[3] = {1, 4, 8};
  std::vector<long long> off(g.N + 1, 0);
  std::vector<int> lists[3];
  int max_nb[3] = {0, 0, 0};
  size_t smem[3] = {0, 0, 0};
  for (int i = 0; i < g.N; ++i) {
    const int nb = (body_start_host[i + 1] - body_start_host[i]) * (kind + 1);
    off[i + 1] = off[i] + (nb <= kMaxBlock ? (long long)nb * nb : 0);
    const int c = nb <= kMaxSingle ? 0 : nb <= kMaxBlock4 ? 1 : nb <= kMaxBlock ? 2 : -1;
    if (c < 0) continue;
    lists[c].push_back(i);
    max_nb[c] = std::max(max_nb[c], nb);
    smem[c] = std::max(smem[c], gj_smem_floats(nb, kCs[c]) * sizeof(float));
  }
  std::vector<int> all;
  for (const auto& l : lists) all.insert(all.end(), l.begin(), l.end());
  cudaError_t e = cudaMemcpyAsync(off_dev, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(fallbacks, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (!all.empty()) {
    e = cudaMemcpyAsync(list_dev, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
  }
  size_t at = 0;
  for (int c = 0; c < 3; ++c) {
    const int count = (int)lists[c].size();
    if (count == 0) continue;
    const int threads = (max_nb[c] + 31) / 32 * 32;
    const int* l = list_dev + at;
    e = c == 0   ? launch_factor<1>(g, kind, alpha, l, count, threads, smem[c], off_dev, blocks, fallbacks, s)
        : c == 1 ? launch_factor<4>(g, kind, alpha, l, count, threads, smem[c], off_dev, blocks, fallbacks, s)
                 : launch_factor<8>(g, kind, alpha, l, count, threads, smem[c], off_dev, blocks, fallbacks, s);
    if (e != cudaSuccess) return e;
    at += count;
  }
  // the host vectors must outlive the asynchronous copies
  return cudaStreamSynchronize(s);
}

cudaError_t bj_apply(const Geo& g, int kind, const long long* off_dev, const bj_t* blocks, VecRef v, double* z,
                     const int* stop, int max_nb, cudaStream_t s, bool f64) {
  const dim3 grid(g.N, (max_nb + kApplyRows - 1) / kApplyRows);
  const size_t nv = (size_t)std::min(max_nb, kMaxBlock);
  if (f64)
    k_bj_apply<true><<<grid, kBA, nv * sizeof(double), s>>>(g, kind, off_dev, blocks, v, z, stop);
  else
    k_bj_apply<false><<<grid, kBA, nv * sizeof(float), s>>>(g, kind, off_dev, blocks, v, z, stop);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bie
