// Quadtree fast multipole method for the pair sums, in complex variables.
//
// With z = x1 + i x2, both kernels reduce to Cauchy sums
//   F_q(z_a) = sum_{b != a} q_b / (z_a - z_b),   F'_q its z-derivative.
// Laplace (Section 3.4): with q = w mu (real) and nu = n1 + i n2 at the target,
//   sum_b q_b (r . n_a)/|r|^2 = Re(nu_a F_q(z_a)).
// Stokes traction (Section 4.3): with q = w (mu1 + i mu2) complex, and
//   S1 = F_q, S2 = -F'_q, S3 = -F'_{q conj(z - c0)}, S6 = F_{conj q} (any c0 fixed for the target),
//   sum_b r (r . q_b)(r . n_a)/|r|^4 =
//     (1/4) [ conj(nu) conj(conj(z_a - c0) S2 - S3) + nu conj(S1) + conj(nu) conj(S6) + nu S1 ],
// an identity of complex algebra (r . m = Re(r conj(m)) for complex r, m).
//
// Uniform quadtree on the bounding square, leaf level L chosen so that a
// non-empty leaf holds about 24-50 nodes.  Expansions in scaled form (powers of
// (z - c)/s), so the translation operators do not depend on the level: 4
// multipole-to-multipole and 4 local-to-local p x p complex matrices, and for
// the multipole-to-local step (offsets -3..3 in each direction) two diagonal
// factors per offset around one real Pascal matrix, built on the host in
// double precision.  Multipole:  F(z) = sum_k a_k s^k / (z - c)^(k+1),
// a_k = sum_j q_j ((z_j - c)/s)^k; local: F(z) = sum_l b_l ((z - c)/s)^l.
// Translations (d = target centre - source centre):
//   M2M  a'_k = sum_{m<=k} C(k,m) 2^-m w^(k-m) a_m,        w = (c_child - c_parent)/S
//   M2L  b_l  = (1/s) sum_k (-1)^l C(k+l,l) D^-(k+l+1) a_k,  D = d/s (integer offset)
//   L2L  b'_m = sum_{l>=m} C(l,m) 2^-m w^(l-m) b_l
// The near field (the 3 x 3 leaves around a target's leaf) is summed directly.
// For the pair sums the S3 channel carries, in every box B, the box-relative
// density q conj(z - c_B)/s_B, so that the combination conj(z_a - c) S2 - S3
// is formed about the target's own leaf centre c: about one global c0 its two
// terms grow with |z_a - c0| and cancel, which costs FP32 expansions their
// accuracy.  The translations add the exact shift terms: M2M takes
// 1/2 a_B + gamma a_0 (gamma = conj(c_child - c_parent)/(2 s_child)), M2L
// a_S - conj(D) a_0, L2L 2 b_P + delta b_0 (delta = conj(c_P - c_C)/s_C).
// Nodes are grouped by leaf with a counting sort whose order inside a leaf is
// the node order, so every sum runs in a fixed order (deterministic results).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"
#include "logtab.cuh"
#include "pair_math.cuh"
#include "reduce.cuh"

namespace bie {

namespace {

constexpr int kMaxP = 64;
constexpr int kB = 64;       // threads per box block (>= p)
constexpr int kChunk = 32;   // points per P2M chunk
constexpr int kMaxNd = 4;    // channels per box

__host__ __device__ inline long long lev_off(int l) { return ((1LL << (2 * l)) - 1) / 3; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}

// The same in FP32 (expansions of the inner solves' operator).
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
template <class T2>
__device__ __forceinline__ T2 cx(double x, double y);
template <>
__device__ __forceinline__ double2 cx<double2>(double x, double y) { return make_double2(x, y); }
template <>
__device__ __forceinline__ float2 cx<float2>(double x, double y) { return make_float2((float)x, (float)y); }

// Tree and expansion buffers of one apply; T2 = double2 (FP64 expansions) or
// float2 (FP32 expansions).  Densities Q stay FP64.
template <class T2>
struct FmmDevT {
  int L, nb, p, nd, M;
  int nlog;           // the first nlog channels carry the logarithm kernel, the rest Cauchy sums
  int cm;             // channel with the box-relative moment density q conj(z - c_B)/s_B (-1: none)
  double x0, y0, D, Dinv;  // bounding square: corner, side, 1/side
  const int* leaf;
  const int* perm;
  const int* start;
  const int* count;   // sources per box (all levels)
  const int* tcount;  // targets per box: boxes that need local expansions
  double2* Q;
  T2* mp;
  T2* lc;
  const T2* ops;
  const float2* Qf = nullptr;  // FP32 expansions: q per source in FP32 (channel 0), from k_fmm_density32
  const float4* cen32 = nullptr;  // FP32 expansions: leaf centres split hi + lo
  float is32 = 0.f, s32 = 0.f;    // FP32 expansions: 1/s and s of a leaf
};
using FmmDev = FmmDevT<double2>;

template <class T2>
__device__ __forceinline__ double2 box_center(const FmmDevT<T2>& f, int l, int bx, int by, double& s) {
  s = ldexp(f.D, -l);  // exact: no division on the (slow) FP64 pipe
  return make_double2(f.x0 + (bx + 0.5) * s, f.y0 + (by + 0.5) * s);
}

// ------------------------------------------------------------------ setup ----
// Bounding square of the body boxes and the total arc length.
constexpr int kBoxT = 256;
__global__ void __launch_bounds__(kBoxT) k_fmm_box(Geo g, double* out) {
  __shared__ double sh[kBoxT / 32];
  double x0 = 1e300, y0 = 1e300, nx1 = 1e300, ny1 = 1e300, len = 0.0;  // nx1, ny1: -max
  for (int i = threadIdx.x; i < g.N; i += kBoxT) {
    const float4 b = g.bbox[i];
    x0 = fmin(x0, (double)b.x);
    y0 = fmin(y0, (double)b.y);
    nx1 = fmin(nx1, -(double)b.z);
    ny1 = fmin(ny1, -(double)b.w);
    len += g.len[i];
  }
  x0 = block_min<kBoxT>(x0, sh);
  y0 = block_min<kBoxT>(y0, sh);
  const double x1 = -block_min<kBoxT>(nx1, sh), y1 = -block_min<kBoxT>(ny1, sh);
  len = block_sum<kBoxT>(len, sh);
  if (threadIdx.x == 0) {
    const double D = fmax(x1 - x0, y1 - y0) * (1.0 + 1e-6) + 1e-12;
    out[0] = x0 - 1e-7 * D;
    out[1] = y0 - 1e-7 * D;
    out[2] = D * (1.0 + 2e-7);
    out[3] = len;
  }
}

__global__ void k_fmm_leaf(Geo g, int L, double x0, double y0, double D, int* leaf, int* cnt) {
  const int nb = 1 << L;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.M; i += gridDim.x * blockDim.x) {
    int ix = (int)((g.x[i] - x0) / D * nb), iy = (int)((g.y[i] - y0) / D * nb);
    ix = min(max(ix, 0), nb - 1);
    iy = min(max(iy, 0), nb - 1);
    const int b = iy * nb + ix;
    leaf[i] = b;
    atomicAdd(&cnt[b], 1);
  }
}

// Exclusive scan of n counts into start[0..n] (one block of 1024 threads).
__global__ void k_fmm_scan(const int* cnt, int n, int* start) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (n + 1023) / 1024;
  const int b0 = t * per, b1 = min(n, b0 + per);
  int s = 0;
  for (int i = b0; i < b1; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int k = 0; k < 1024; ++k) {
      const int v = part[k];
      part[k] = acc;
      acc += v;
    }
    start[n] = acc;
  }
  __syncthreads();
  int acc = part[t];
  for (int i = b0; i < b1; ++i) {
    start[i] = acc;
    acc += cnt[i];
  }
}

__global__ void k_fmm_scatter(int M, const int* leaf, const int* start, int* cursor, int* tmp) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
    const int b = leaf[i];
    tmp[start[b] + atomicAdd(&cursor[b], 1)] = i;
  }
}

// Within each leaf, put the nodes in increasing node order (rank by counting).
__global__ void k_fmm_order(const int* start, const int* tmp, int* perm) {
  const int b = blockIdx.x;
  const int s0 = start[b], n = start[b + 1] - s0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int v = tmp[s0 + j];
    int rank = 0;
    for (int k = 0; k < n; ++k) rank += tmp[s0 + k] < v;
    perm[s0 + rank] = v;
  }
}

// Points per box on every level: leaves from start, parents from children.
__global__ void k_fmm_leaf_counts(const int* start, int nleaf, int* count_leaf) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nleaf; b += gridDim.x * blockDim.x)
    count_leaf[b] = start[b + 1] - start[b];
}
__global__ void k_fmm_parent_counts(int l, int* count) {
  const int n = 1 << l;
  const long long off = lev_off(l), offc = lev_off(l + 1);
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n * n; b += gridDim.x * blockDim.x) {
    const int bx = b % n, by = b / n;
    const int nc = 2 * n;
    int s = 0;
    for (int c = 0; c < 4; ++c) s += count[offc + (2 * by + (c >> 1)) * nc + 2 * bx + (c & 1)];
    count[off + b] = s;
  }
}

// ------------------------------------------------------------------ apply ----
// Densities: Laplace q = sw v (real); Stokes q = sw (v1 + i v2), conj(q),
// q conj(z - c0) with c0 the centre of the bounding square (the Stokes
// combination cancels conj(z_a) S2 against S3, so smaller |z - c0| keeps the
// expansion error of S3 small).
__global__ void k_fmm_density(Geo g, int nd, double cx0, double cy0, VecRef vr, const double* __restrict__ sscale,
                              double2* Q, const int* stop) {
  if (stop && *stop) return;
  const double* v = vr.ptr();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.M; i += gridDim.x * blockDim.x) {
    if (nd == 1) {
      Q[i] = make_double2(sscale[i] * v[i], 0.0);
    } else {
      const double2 q = make_double2(sscale[i] * v[2 * i], sscale[i] * v[2 * i + 1]);
      Q[3 * i] = q;
      Q[3 * i + 1] = cconj(q);
      Q[3 * i + 2] = cmul(q, make_double2(g.x[i] - cx0, -(g.y[i] - cy0)));
    }
  }
}

// The P2M terms of one chunk of m sources: output e = d p + k (channel d,
// coefficient k) is owned by thread e mod kB, which adds its terms in source
// order (fixed: deterministic).  All p nd outputs run in parallel (p = 18,
// nd = 3: 54 of 64 threads), each a chain of m complex multiply-adds.
constexpr int kP2MAcc = (kMaxNd * kMaxP + kB - 1) / kB;  // outputs a thread keeps
template <class T2>
__device__ __forceinline__ void p2m_chunk(T2* acc, const T2* pw, const T2* qs, int p, int nd, int m) {
  const int np = p * nd;
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u) {
    const int e = threadIdx.x + u * kB;
    if (e < np) {
      const int d = e / p, k = e - d * p;
      const T2* pk = pw + k * (kChunk + 1);
      T2 a = acc[u];
      for (int j = 0; j < m; ++j) cfma(a, pk[j], qs[j * nd + d]);
      acc[u] = a;
    }
  }
}

// The FP32 operator's strengths: q = sqrt(w) v per source in FP32 (Laplace:
// (q, 0); Stokes: the complex density).  The other channels (conj(q) and the
// leaf-relative moment density) are formed where they are used, so the FP32
// passes read 8 bytes a source and convert nothing from FP64.
__global__ void k_fmm_density32(Geo g, int nd, VecRef vr, const double* __restrict__ sscale, float2* Qf,
                                const int* stop) {
  if (stop && *stop) return;
  const double* v = vr.ptr();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.M; i += gridDim.x * blockDim.x) {
    if (nd == 1)
      Qf[i] = make_float2((float)(sscale[i] * v[i]), 0.f);
    else
      Qf[i] = make_float2((float)(sscale[i] * v[2 * i]), (float)(sscale[i] * v[2 * i + 1]));
  }
}

// Leaf centres split as float hi + lo, once per tree (FP64 arithmetic here,
// so that the FP32 passes form u = (z - c)/s from the hi/lo split of z in
// FP32 with no FP64 instruction: z_hi - c_hi is exact for a node inside the
// leaf unless |z| is of the order of s).
__global__ void k_fmm_leaf_centers(int nb, double x0, double y0, double s, float4* cen) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb * nb; b += gridDim.x * blockDim.x) {
    const double cx = x0 + (b % nb + 0.5) * s, cy = y0 + (b / nb + 0.5) * s;
    const float hx = (float)cx, hy = (float)cy;
    cen[b] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
  }
}

// The block's leaf centre split (x_h, y_h, x_l, y_l), 1/s and s in shared memory.
__device__ __forceinline__ void leaf_center32(const FmmDevT<float2>& f, int b, float* cen) {
  if (threadIdx.x == 0) {
    const float4 c = f.cen32[b];
    cen[0] = c.x;
    cen[1] = c.y;
    cen[2] = c.z;
    cen[3] = c.w;
    cen[4] = f.is32;
    cen[5] = f.s32;
  }
}

// P2M of the FP32 expansions (inner solves) with no FP64 instruction per
// source: positions from the hi/lo split, strengths from k_fmm_density32.
__global__ void __launch_bounds__(kB) k_fmm_p2m32(FmmDevT<float2> f, Geo g, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* pw = reinterpret_cast<float2*>(smraw);  // [p][kChunk + 1]
  float2* qs = pw + f.p * (kChunk + 1);            // [kChunk][nd]
  __shared__ float cen[6];
  const int b = blockIdx.x;
  const long long box = lev_off(f.L) + b;
  const int s0 = f.start[b], n = f.start[b + 1] - s0;
  if (n == 0) return;
  leaf_center32(f, b, cen);
  __syncthreads();
  const int t = threadIdx.x;
  float2 acc[kP2MAcc];
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u) acc[u] = make_float2(0.f, 0.f);
  for (int ch = 0; ch < n; ch += kChunk) {
    const int m = min(kChunk, n - ch);
    if (t < m) {
      const int i = f.perm[s0 + ch + t];
      const float4 P = g.pf[i];
      const float2 u = make_float2(((P.x - cen[0]) + (P.z - cen[2])) * cen[4], ((P.y - cen[1]) + (P.w - cen[3])) * cen[4]);
      float2 w = make_float2(1.f, 0.f);
      for (int k = 0; k < f.p; ++k) {
        pw[k * (kChunk + 1) + t] = w;
        w = cmul(w, u);
      }
      const float2 q = f.Qf[i];
      qs[t * f.nd] = q;
      if (f.nd == 3) {
        qs[t * 3 + 1] = make_float2(q.x, -q.y);
        // channel cm = 2: q conj(u), the leaf-relative moment density
        qs[t * 3 + 2] = make_float2(q.x * u.x + q.y * u.y, q.y * u.x - q.x * u.y);
      }
    }
    __syncthreads();
    p2m_chunk(acc, pw, qs, f.p, f.nd, m);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u)
    if (t + u * kB < f.nd * f.p) f.mp[box * f.nd * f.p + t + u * kB] = acc[u];
}

// P2M on the leaves: a_k = sum_j q_j u_j^k, u = (z - c)/s.
template <class T2>
__global__ void __launch_bounds__(kB) k_fmm_p2m(FmmDevT<T2> f, Geo g, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  T2* pw = sm;                       // [p][kChunk + 1]
  T2* qs = sm + f.p * (kChunk + 1);  // [kChunk][nd]
  const int b = blockIdx.x;
  const long long box = lev_off(f.L) + b;
  const int s0 = f.start[b], n = f.start[b + 1] - s0;
  if (n == 0) return;
  double s;
  const double2 c = box_center(f, f.L, b % f.nb, b / f.nb, s);
  const int t = threadIdx.x;
  T2 acc[kP2MAcc];
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u) acc[u] = cx<T2>(0.0, 0.0);
  for (int ch = 0; ch < n; ch += kChunk) {
    const int m = min(kChunk, n - ch);
    if (t < kChunk) {
      if (t < m) {
        const int i = f.perm[s0 + ch + t];
        const double is = ldexp(f.Dinv, f.L);
        const T2 u = cx<T2>((g.x[i] - c.x) * is, (g.y[i] - c.y) * is);
        T2 w = cx<T2>(1.0, 0.0);
        for (int k = 0; k < f.p; ++k) {
          pw[k * (kChunk + 1) + t] = w;
          w = cmul(w, u);
        }
        for (int d = 0; d < f.nd; ++d) {
          const double2 q = f.Q[(long long)i * f.nd + (d == f.cm ? 0 : d)];
          // channel cm: q conj(u), the leaf-relative moment density
          qs[t * f.nd + d] = d == f.cm ? cx<T2>(q.x * (double)u.x + q.y * (double)u.y,
                                                q.y * (double)u.x - q.x * (double)u.y)
                                       : cx<T2>(q.x, q.y);
        }
      }
    }
    __syncthreads();
    p2m_chunk(acc, pw, qs, f.p, f.nd, m);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u)
    if (t + u * kB < f.nd * f.p) f.mp[box * f.nd * f.p + t + u * kB] = acc[u];
}

// M2M into level l (parents) from level l + 1.  Per child, its multipoles and
// the translation matrix are staged in shared memory (coalesced, one round
// trip each); thread e < nd p computes coefficient e % p of channel e / p
// (its terms in the order m = 0..k), summed over the children in order.
constexpr int kAccPer = (kMaxNd * kMaxP + kB - 1) / kB;  // outputs a thread keeps

template <class T2>
__global__ void __launch_bounds__(kB) k_fmm_m2m(FmmDevT<T2> f, int l, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);  // [nd][p]
  T2* so = sm + f.nd * f.p;               // [p][p] the child's M2M matrix, [in][out]
  const int n = 1 << l;
  const int b = blockIdx.x, bx = b % n, by = b / n;
  const long long box = lev_off(l) + b;
  if (f.count[box] == 0) return;
  const int t = threadIdx.x, np = f.nd * f.p, pp = f.p * f.p;
  T2 acc[kAccPer];
#pragma unroll
  for (int u = 0; u < kAccPer; ++u) acc[u] = cx<T2>(0.0, 0.0);
  for (int c = 0; c < 4; ++c) {
    const long long child = lev_off(l + 1) + (2 * by + (c >> 1)) * (2 * n) + 2 * bx + (c & 1);
    if (f.count[child] == 0) continue;  // uniform over the block
    __syncthreads();
    for (int e = t; e < np; e += kB) sm[e] = f.mp[child * np + e];
    for (int e = t; e < pp; e += kB) so[e] = f.ops[(long long)c * pp + e];
    __syncthreads();
    if (f.cm >= 0) {
      // child moment density relative to the parent centre: 1/2 rho_C + gamma rho_0,
      // gamma = conj(c_C - c_P)/(2 s_C)
      const T2 gam = cx<T2>(0.5 * ((c & 1) - 0.5), -0.5 * ((c >> 1) - 0.5));
      for (int m = t; m < f.p; m += kB) {
        T2 v = cx<T2>(0.5 * (double)sm[f.cm * f.p + m].x, 0.5 * (double)sm[f.cm * f.p + m].y);
        cfma(v, gam, sm[m]);
        sm[f.cm * f.p + m] = v;
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < kAccPer; ++u) {
      const int e = t + u * kB;
      if (e < np) {
        const int d = e / f.p, k = e % f.p;
        for (int m = 0; m <= k; ++m) cfma(acc[u], so[m * f.p + k], sm[d * f.p + m]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < kAccPer; ++u) {
    const int e = t + u * kB;
    if (e < np) f.mp[box * np + e] = acc[u];
  }
}

// M2L for the target boxes of all levels 2..L (one block per box), through
// a factorisation of the translation operators (d = D s, D the integer
// offset of the target centre from the source centre in box sides):
//   Cauchy:    T_D[l][k] = (-1)^l C(k+l, l) D^-(k+l+1) = beta_l(D) P[l][k] alpha_k(D),
//              P[l][k] = C(k+l, l),  alpha_k = D^-k,  beta_l = (-1)^l D^-(l+1);
//   logarithm: T^log_D[l][k] = beta_l(D) P^log[l][k] alpha_k(D) for k >= 1,
//              P^log[l][k] = C(k+l-1, l),  alpha_k = D^-k / k,  beta_l = -(-1)^l D^-l,
//              and the a_0 column gamma_l(D) = log D (l = 0), (-1)^(l+1) D^-l / l (l >= 1).
// P is real and the same for every offset, so a box pair costs 2 p^2 real
// multiply-adds (the Pascal matrix times a complex vector) and 8 p for the
// two diagonal scalings, against 4 p^2 for a complex p x p operator.  Cauchy
// channels carry 1/s; logarithm channels add a_0 log(s) on b_0 (the level's
// share of log d = log D + log s).
//
// One warp finds the interaction list (at most 27 boxes, in row-major order
// of the parent's 6 x 6 neighbourhood); the sources' multipoles are staged
// in shared memory already scaled by alpha, U[q][d][k] (q padded with zeros
// to a multiple of 4); thread e < p nd computes coefficient l = e % p of
// channel d = e / p over four sources at a time (four independent chains).
// PM > 0: the thread's Pascal row is held in registers and U is zero-padded
// to PM coefficients (p <= PM); PM = 0: the Pascal matrices are read from
// shared memory, transposed, for any p.
constexpr int kListPad = 28;  // the 27 interaction-list boxes rounded up to the 4-source step
constexpr int kOffs = 49;     // offsets -3..3 x -3..3 (the 3 x 3 near ones unused)

// Layout of the operator table of order p (complex entries): M2M and L2L
// matrices [op][in][out], then the M2L factors alpha[2][49][p], beta[2][49][p],
// gamma[49][p] and the Pascal matrices [2][k][l] (real, in the real parts);
// type 0 = Cauchy, 1 = logarithm, offset index (Dx + 3) + 7 (Dy + 3).
__host__ __device__ inline long long tab_alpha(int p) { return 8LL * p * p; }
__host__ __device__ inline long long tab_beta(int p) { return tab_alpha(p) + 2LL * kOffs * p; }
__host__ __device__ inline long long tab_gamma(int p) { return tab_beta(p) + 2LL * kOffs * p; }
__host__ __device__ inline long long tab_pascal(int p) { return tab_gamma(p) + (long long)kOffs * p; }
__host__ __device__ inline long long tab_size(int p) { return tab_pascal(p) + 2LL * p * p; }

// w += (pp.x u.x, pp.y u.y): a real factor (duplicated in pp) times a complex value
__device__ __forceinline__ void rfma(float2& w, float2 pp, float2 u) { w = __ffma2_rn(pp, u, w); }
__device__ __forceinline__ void rfma(double2& w, double2 pp, double2 u) {
  w.x = fma(pp.x, u.x, w.x);
  w.y = fma(pp.y, u.y, w.y);
}

template <class T2, int PM>
__global__ void __launch_bounds__(256) k_fmm_m2l(FmmDevT<T2> f, const int* stop) {
  using R = decltype(T2{}.x);
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_src[kListPad];
  __shared__ int s_off[kListPad];
  __shared__ T2 s_a0[kListPad][kMaxNd];  // raw a_0 of the logarithm channels
  __shared__ int s_cnt;
  long long gb = blockIdx.x + lev_off(2);
  int l = 2;
  while (l < f.L && gb >= lev_off(l + 1)) ++l;
  if (f.tcount[gb] == 0) return;
  const int p = f.p, nd = f.nd, pk = PM > 0 ? PM : p;
  const int n = 1 << l;
  const int b = (int)(gb - lev_off(l)), bx = b % n, by = b / n;
  const int px = bx >> 1, py = by >> 1;
  const int tid = threadIdx.x;
  if (tid < 32) {
    int base = 0;
    for (int r = 0; r < 2; ++r) {
      const int c = r * 32 + tid;
      const int sx = 2 * px - 2 + c % 6, sy = 2 * py - 2 + c / 6;
      bool ok = c < 36 && sx >= 0 && sy >= 0 && sx < n && sy < n && !(abs(sx - bx) <= 1 && abs(sy - by) <= 1);
      const long long src = lev_off(l) + (long long)sy * n + sx;
      if (ok) ok = f.count[src] != 0;
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int pos = base + __popc(m & ((1u << tid) - 1u));
        s_src[pos] = sy * n + sx;
        s_off[pos] = (bx - sx + 3) + 7 * (by - sy + 3);
      }
      base += __popc(m);
    }
    if (tid == 0) s_cnt = base;
  }
  __syncthreads();
  const int cnt = s_cnt, cnt4 = (cnt + 3) & ~3;
  T2* U = reinterpret_cast<T2*>(smraw);  // [cnt4][nd][pk]
  R* Pt = reinterpret_cast<R*>(U + (long long)kListPad * nd * pk);  // PM = 0: [type][k][l]
  const T2* alpha = f.ops + tab_alpha(p);
  const T2* beta = f.ops + tab_beta(p);
  const T2* gamma = f.ops + tab_gamma(p);
  const T2* pas = f.ops + tab_pascal(p);
  const int ntype = f.nlog > 0 ? 2 : 1;
  if (PM == 0)
    for (int e = tid; e < ntype * p * p; e += blockDim.x) {
      const int t = e / (p * p), r = e % (p * p);
      Pt[e] = pas[(long long)(f.nlog > 0 ? t : 0) * p * p + r].x;
    }
  const int per = nd * pk;
  // a thread keeps its (channel, coefficient) and walks the sources
  for (int dk = tid; dk < per; dk += blockDim.x) {
    const int d = dk / pk, k = dk % pk;
    const int ty = d < f.nlog ? 1 : 0;
    const T2* al = alpha + (long long)ty * kOffs * p + k;
#pragma unroll 4
    for (int q = 0; q < cnt4; ++q) {
      T2 u = cx<T2>(0.0, 0.0);
      if (q < cnt && k < p) {
        const T2* a = f.mp + ((lev_off(l) + s_src[q]) * nd) * p;
        const int oi = s_off[q];
        T2 v = a[d * p + k];
        if (d == f.cm) {
          // source moment density relative to the target centre: rho_S - conj(D) rho_0
          cfma(v, cx<T2>((double)(3 - oi % 7), (double)(oi / 7 - 3)), a[k]);
        }
        if (ty == 1 && k == 0) s_a0[q][d] = v;
        u = cmul(al[(long long)oi * p], v);
      }
      U[q * per + dk] = u;
    }
  }
  __syncthreads();
  const double inv_s = ldexp(f.Dinv, l);
  for (int e = tid; e < nd * p; e += blockDim.x) {
    const int d = e / p, t = e % p;
    const int ty = d < f.nlog ? 1 : 0;
    const int tp = f.nlog > 0 ? ty : 0;  // Pascal slot of this channel
    // log s (s = D 2^-l), on b_0 of the logarithm channels only
    const R logs = (ty == 1 && t == 0) ? (R)(log(f.D) - l * 0.69314718055994530942) : (R)0;
    T2 prow[PM > 0 ? PM : 1];
    if (PM > 0) {
#pragma unroll
      for (int k = 0; k < (PM > 0 ? PM : 1); ++k) {
        const R v = k < p ? pas[((long long)ty * p + k) * p + t].x : (R)0;
        prow[k] = cx<T2>((double)v, (double)v);
      }
    }
    T2 acc = cx<T2>(0.0, 0.0);
    for (int q0 = 0; q0 < cnt; q0 += 4) {
      T2 w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = cx<T2>(0.0, 0.0);
      const T2* u = U + ((long long)q0 * nd + d) * pk;
      if (PM > 0) {
#pragma unroll
        for (int k = 0; k < (PM > 0 ? PM : 1); ++k)
#pragma unroll
          for (int j = 0; j < 4; ++j) rfma(w[j], prow[k], u[(long long)j * per + k]);
      } else {
        const R* pt = Pt + (long long)tp * p * p + t;
        for (int k = 0; k < p; ++k) {
          const R pv = pt[(long long)k * p];
          const T2 pp = cx<T2>((double)pv, (double)pv);
#pragma unroll
          for (int j = 0; j < 4; ++j) rfma(w[j], pp, u[(long long)j * per + k]);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (q0 + j < cnt) {
          const int oi = s_off[q0 + j];
          cfma(acc, beta[((long long)ty * kOffs + oi) * p + t], w[j]);
          if (ty == 1) {
            T2 gm = gamma[(long long)oi * p + t];
            if (t == 0) gm.x += logs;
            cfma(acc, gm, s_a0[q0 + j][d]);
          }
        }
      }
    }
    // Cauchy channels carry 1/s; in the precision of the expansions
    const R sc = ty == 1 ? (R)1 : (R)inv_s;
    acc.x *= sc;
    acc.y *= sc;
    f.lc[(gb * nd + d) * p + t] = acc;
  }
}

// Shared memory of one M2L block: the staged sources and, for PM = 0, the
// transposed Pascal matrices.
template <class T2>
size_t m2l_smem(int p, int nd, int nlog, int pm) {
  const int pk = pm > 0 ? pm : p;
  size_t b = (size_t)kListPad * nd * pk * sizeof(T2);
  if (pm == 0) b += (size_t)(nlog > 0 ? 2 : 1) * p * p * sizeof(decltype(T2{}.x));
  return b;
}

// ---- float-float M2L: the residual operator of the float-float refinement ----
// The multipoles (FP64) are split once into float-float pairs hi + lo
// (k_fmm_mp_ff); the factorised M2L then runs on the FP32 pipe in pairs of
// lanes (real, imaginary): a Pascal entry times a source coefficient is an
// exact FP32 product plus its error term and the cross terms (about 48
// significant bits), accumulated with an error-free sum and renormalised at
// every step, and the diagonal factors alpha and beta are float-float splits
// of the FP64 tables.  Relative rounding about 2^-48 per operation, against
// 2^-53 in FP64, on a pipe that issues many times more operations; the local
// expansions are written back in FP64.  Cauchy channels only (the pair sums).
// Complex float-float values are float4 (re_hi, im_hi, re_lo, im_lo).
__global__ void k_fmm_mp_ff(const double2* __restrict__ mp, long long n, float4* __restrict__ mpff) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = mp[i];
    const float rh = (float)a.x, ih = (float)a.y;
    mpff[i] = make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
  }
}

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// (ph, pl) = (ah + al)(bh + bl) lane-wise: exact leading product, its error
// and the cross terms
__device__ __forceinline__ void ff_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2& ph, float2& pl) {
  ph = __fmul2_rn(ah, bh);
  pl = __ffma2_rn(ah, bh, neg2(ph));
  pl = __ffma2_rn(ah, bl, pl);
  pl = __ffma2_rn(al, bh, pl);
}

// (sh, sl) += (ph, pl) lane-wise: error-free sum of the leading parts, the
// low parts added, renormalised
__device__ __forceinline__ void ff_acc2(float2& sh, float2& sl, float2 ph, float2 pl) {
  const float2 s = __fadd2_rn(sh, ph);
  const float2 bb = __fadd2_rn(s, neg2(sh));
  const float2 e = __fadd2_rn(__fadd2_rn(sh, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(ph, neg2(bb)));
  const float2 t = __fadd2_rn(e, __fadd2_rn(sl, pl));
  sh = __fadd2_rn(s, t);
  sl = __fadd2_rn(t, neg2(__fadd2_rn(sh, neg2(s))));
}

// (sh, sl) += a b, complex float-float: a = (ah, al), b = (bh, bl) as
// (re, im) lane pairs
__device__ __forceinline__ void ff_cfma(float2& sh, float2& sl, float2 ah, float2 al, float2 bh, float2 bl) {
  float2 xh, xl, yh, yl;
  // (a_re b_re, a_re b_im) + (-a_im b_im, a_im b_re)
  ff_mul2(make_float2(ah.x, ah.x), make_float2(al.x, al.x), bh, bl, xh, xl);
  ff_mul2(make_float2(ah.y, ah.y), make_float2(al.y, al.y), make_float2(-bh.y, bh.x), make_float2(-bl.y, bl.x), yh,
          yl);
  ff_acc2(sh, sl, xh, xl);
  ff_acc2(sh, sl, yh, yl);
}

// Complex float-float values as (re, im) lane pairs: h the leading parts, l
// the trailing ones.
struct cff {
  float2 h, l;
};
__device__ __forceinline__ cff cff_zero() { return cff{make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ cff cff_load(float4 v) { return cff{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ cff cff_split(double re, double im) {
  const float rh = (float)re, ih = (float)im;
  return cff{make_float2(rh, ih), make_float2((float)(re - (double)rh), (float)(im - (double)ih))};
}
__device__ __forceinline__ double2 cff_to(cff a) {
  return make_double2((double)a.h.x + (double)a.l.x, (double)a.h.y + (double)a.l.y);
}
__device__ __forceinline__ cff cff_conj(cff a) {
  return cff{make_float2(a.h.x, -a.h.y), make_float2(a.l.x, -a.l.y)};
}
__device__ __forceinline__ cff cff_neg(cff a) { return cff{neg2(a.h), neg2(a.l)}; }
// acc + a b
__device__ __forceinline__ cff cff_fma(cff acc, cff a, cff b) {
  ff_cfma(acc.h, acc.l, a.h, a.l, b.h, b.l);
  return acc;
}
// a (sh + sl), a real float-float factor
__device__ __forceinline__ cff cff_scale(cff a, float sh, float sl) {
  cff r;
  ff_mul2(make_float2(sh, sh), make_float2(sl, sl), a.h, a.l, r.h, r.l);
  return r;
}

__device__ __forceinline__ float4 cff_store(cff a) { return make_float4(a.h.x, a.h.y, a.l.x, a.l.y); }

// P2M of the float-float residual's FMM and of the float-float solves'
// output FMM (FP64 expansions): the powers of u and the sums in float-float
// on the FP32 pipe (about 48 bits, what the
// float-float residual certifies; GB300 runs FP64 multiply-adds at two lanes
// a clock per SM).  Layout and term order as k_fmm_p2m: output e = d p + k
// on thread e mod kB, sources in order.
__global__ void __launch_bounds__(kB) k_fmm_p2m_ff(FmmDevT<double2> f, Geo g, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* pw = reinterpret_cast<float4*>(smraw);  // [p][kChunk + 1] u^k as (re_h, im_h, re_l, im_l)
  float4* qs = pw + f.p * (kChunk + 1);            // [kChunk][nd]
  const int b = blockIdx.x;
  const long long box = lev_off(f.L) + b;
  const int s0 = f.start[b], n = f.start[b + 1] - s0;
  if (n == 0) return;
  const int t = threadIdx.x, np = f.p * f.nd;
  cff acc[kP2MAcc];
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u) acc[u] = cff_zero();
  for (int ch = 0; ch < n; ch += kChunk) {
    const int m = min(kChunk, n - ch);
    if (t < m) {
      double s;
      const double2 c = box_center(f, f.L, b % f.nb, b / f.nb, s);
      const int i = f.perm[s0 + ch + t];
      const double is = ldexp(f.Dinv, f.L);
      const cff U = cff_split((g.x[i] - c.x) * is, (g.y[i] - c.y) * is);
      cff w = cff_split(1.0, 0.0);
      for (int k = 0; k < f.p; ++k) {
        pw[k * (kChunk + 1) + t] = cff_store(w);
        w = cff_fma(cff_zero(), w, U);
      }
      for (int d = 0; d < f.nd; ++d) {
        // channel cm: q_0 conj(u), the leaf-relative moment density
        const double2 q = f.Q[(long long)i * f.nd + (d == f.cm ? 0 : d)];
        const cff qd = cff_split(q.x, q.y);
        qs[t * f.nd + d] = cff_store(d == f.cm ? cff_fma(cff_zero(), qd, cff_conj(U)) : qd);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kP2MAcc; ++u) {
      const int e = t + u * kB;
      if (e < np) {
        const int d = e / f.p, k = e - d * f.p;
        const float4* pk = pw + k * (kChunk + 1);
        cff a = acc[u];
        for (int j = 0; j < m; ++j) a = cff_fma(a, cff_load(pk[j]), cff_load(qs[j * f.nd + d]));
        acc[u] = a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kP2MAcc; ++u)
    if (t + u * kB < np) f.mp[box * np + t + u * kB] = cff_to(acc[u]);
}

// Tables of order p: alpha[2][49][p], beta[2][49][p], gamma[49][p] (float4;
// type 0 Cauchy, 1 logarithm, as tab_alpha..tab_gamma), then the Pascal
// matrices [2][k][l] (float2 hi, lo).
__host__ __device__ inline long long fftab_beta(int p) { return 2LL * kOffs * p; }
__host__ __device__ inline long long fftab_gamma(int p) { return 4LL * kOffs * p; }
__host__ __device__ inline long long fftab_pascal(int p) { return 5LL * kOffs * p; }  // in float4 units
__host__ __device__ inline long long fftab_floats(int p) { return 20LL * kOffs * p + 4LL * p * p; }

constexpr int kBFF = 128;

__global__ void __launch_bounds__(kBFF) k_fmm_m2l_ff(FmmDev f, const float4* __restrict__ mpff,
                                                     const float* __restrict__ tab, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_src[kListPad];
  __shared__ int s_off[kListPad];
  __shared__ float4 s_a0[kListPad][kMaxNd];  // a_0 of the logarithm channels
  __shared__ int s_cnt;
  long long gb = blockIdx.x + lev_off(2);
  int l = 2;
  while (l < f.L && gb >= lev_off(l + 1)) ++l;
  if (f.tcount[gb] == 0) return;
  const int p = f.p, nd = f.nd;
  const int n = 1 << l;
  const int b = (int)(gb - lev_off(l)), bx = b % n, by = b / n;
  const int px = bx >> 1, py = by >> 1;
  const int tid = threadIdx.x;
  if (tid < 32) {
    int base = 0;
    for (int r = 0; r < 2; ++r) {
      const int c = r * 32 + tid;
      const int sx = 2 * px - 2 + c % 6, sy = 2 * py - 2 + c / 6;
      bool ok = c < 36 && sx >= 0 && sy >= 0 && sx < n && sy < n && !(abs(sx - bx) <= 1 && abs(sy - by) <= 1);
      const long long src = lev_off(l) + (long long)sy * n + sx;
      if (ok) ok = f.count[src] != 0;
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (ok) {
        const int pos = base + __popc(m & ((1u << tid) - 1u));
        s_src[pos] = sy * n + sx;
        s_off[pos] = (bx - sx + 3) + 7 * (by - sy + 3);
      }
      base += __popc(m);
    }
    if (tid == 0) s_cnt = base;
  }
  __syncthreads();
  const int cnt = s_cnt, cnt4 = (cnt + 3) & ~3;
  float4* U = reinterpret_cast<float4*>(smraw);  // [cnt4][nd][p]
  const float4* alpha = reinterpret_cast<const float4*>(tab);
  const float4* beta = alpha + fftab_beta(p);
  const float4* gamma = alpha + fftab_gamma(p);
  const float2* pas = reinterpret_cast<const float2*>(alpha + fftab_pascal(p));
  const int per = nd * p;
  // a thread keeps its (channel, coefficient) and walks the sources
  for (int dk = tid; dk < per; dk += blockDim.x) {
    const int d = dk / p, k = dk % p;
    const int ty = d < f.nlog ? 1 : 0;
    const float4* alk = alpha + (long long)ty * kOffs * p + k;
#pragma unroll 2
    for (int q = 0; q < cnt4; ++q) {
      float2 uh = make_float2(0.f, 0.f), ul = uh;
      if (q < cnt) {
        const float4* a = mpff + ((lev_off(l) + s_src[q]) * nd) * p;
        const int oi = s_off[q];
        const float4 v = a[d * p + k];
        float2 vh = make_float2(v.x, v.y), vl = make_float2(v.z, v.w);
        if (d == f.cm) {
          // source moment density relative to the target centre: rho_S - conj(D) rho_0
          const float4 a0 = a[k];
          ff_cfma(vh, vl, make_float2((float)(3 - oi % 7), (float)(oi / 7 - 3)), make_float2(0.f, 0.f),
                  make_float2(a0.x, a0.y), make_float2(a0.z, a0.w));
        }
        if (ty == 1 && k == 0) s_a0[q][d] = make_float4(vh.x, vh.y, vl.x, vl.y);
        const float4 al = alk[(long long)oi * p];
        ff_cfma(uh, ul, make_float2(al.x, al.y), make_float2(al.z, al.w), vh, vl);
      }
      U[q * per + dk] = make_float4(uh.x, uh.y, ul.x, ul.y);
    }
  }
  __syncthreads();
  const double inv_s = ldexp(f.Dinv, l);
  for (int e = tid; e < per; e += blockDim.x) {
    const int d = e / p, t = e % p;
    const int ty = d < f.nlog ? 1 : 0;
    // log s (s = D 2^-l) on b_0 of the logarithm channels, split hi + lo
    float lsh = 0.f, lsl = 0.f;
    if (ty == 1 && t == 0) {
      const double ls = log(f.D) - l * 0.69314718055994530942;
      lsh = (float)ls;
      lsl = (float)(ls - (double)lsh);
    }
    const float2* pcol = pas + (long long)ty * p * p + t;
    float2 ah = make_float2(0.f, 0.f), al = ah;
    for (int q0 = 0; q0 < cnt; q0 += 4) {
      float2 sh[4], sl[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) sh[j] = sl[j] = make_float2(0.f, 0.f);
      const float4* u = U + (long long)q0 * per + d * p;
      for (int k = 0; k < p; ++k) {
        const float2 pv = __ldg(pcol + (long long)k * p);
        const float2 PH = make_float2(pv.x, pv.x), PL = make_float2(pv.y, pv.y);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 uv = u[(long long)j * per + k];
          float2 ph, pl;
          ff_mul2(PH, PL, make_float2(uv.x, uv.y), make_float2(uv.z, uv.w), ph, pl);
          ff_acc2(sh[j], sl[j], ph, pl);
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (q0 + j < cnt) {
          const int oi = s_off[q0 + j];
          const float4 be = beta[((long long)ty * kOffs + oi) * p + t];
          ff_cfma(ah, al, make_float2(be.x, be.y), make_float2(be.z, be.w), sh[j], sl[j]);
          if (ty == 1) {
            // the a_0 column: gamma_l(D) a_0, and log s on b_0
            float4 gm = gamma[(long long)oi * p + t];
            float2 gh = make_float2(gm.x, gm.y), gl = make_float2(gm.z, gm.w);
            ff_acc2(gh, gl, make_float2(lsh, 0.f), make_float2(lsl, 0.f));
            const float4 a0 = s_a0[q0 + j][d];
            ff_cfma(ah, al, gh, gl, make_float2(a0.x, a0.y), make_float2(a0.z, a0.w));
          }
        }
      }
    }
    // Cauchy channels carry 1/s
    const double sc = ty == 1 ? 1.0 : inv_s;
    f.lc[(gb * nd + d) * p + t] =
        make_double2(((double)ah.x + (double)al.x) * sc, ((double)ah.y + (double)al.y) * sc);
  }
}

// L2L from level l to the children at level l + 1 (added to their M2L part):
// the parent's local expansion and the child's L2L matrix staged in shared
// memory; thread e < nd p updates coefficient e % p of channel e / p (terms
// in the order m = k..p-1).
template <class T2>
__global__ void __launch_bounds__(kB) k_fmm_l2l(FmmDevT<T2> f, int l, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);  // [nd][p]
  T2* so = sm + f.nd * f.p;               // [p][p] the L2L matrix, [in][out]
  const int nc = 2 << l;
  const int b = blockIdx.x, bx = b % nc, by = b / nc;
  const long long child = lev_off(l + 1) + b;
  if (f.tcount[child] == 0) return;
  const long long parent = lev_off(l) + (by >> 1) * (nc >> 1) + (bx >> 1);
  const int c = (bx & 1) + 2 * (by & 1);
  const int t = threadIdx.x, np = f.nd * f.p, pp = f.p * f.p;
  for (int e = t; e < np; e += kB) sm[e] = f.lc[parent * np + e];
  for (int e = t; e < pp; e += kB) so[e] = f.ops[(long long)(4 + c) * pp + e];
  __syncthreads();
  if (f.cm >= 0) {
    // moment density relative to the child centre: 2 rho_P + delta rho_0,
    // delta = conj(c_P - c_C)/s_C
    const T2 del = cx<T2>(-((c & 1) - 0.5), (c >> 1) - 0.5);
    for (int m = t; m < f.p; m += kB) {
      T2 v = cx<T2>(2.0 * (double)sm[f.cm * f.p + m].x, 2.0 * (double)sm[f.cm * f.p + m].y);
      cfma(v, del, sm[m]);
      sm[f.cm * f.p + m] = v;
    }
    __syncthreads();
  }
  for (int e = t; e < np; e += kB) {
    const int d = e / f.p, k = e % f.p;
    T2 acc = f.lc[child * np + e];
    for (int m = k; m < f.p; ++m) cfma(acc, so[m * f.p + k], sm[d * f.p + m]);
    f.lc[child * np + e] = acc;
  }
}

// Local expansion and near field at every node of a leaf, then the kernel's
// combination into the pair-sum partial (Laplace scalar / Stokes 2-vector).
// NEARP = 0: the near field enters the FP64 Cauchy sums.  NEARP = 1 (FP32)
// and 2 (float-float): the far part is combined into the kernel value in
// FP64 and the near field is summed as the real kernel with the pair
// arithmetic of the direct sums (exact leading coordinate differences), so
// the accuracy follows the operator that uses it: FP32 for the inner solves,
// float-float for residuals.
constexpr int kNearChunk = 256;  // near-field sources staged per round

template <class T2, int NEARP>
__global__ void __launch_bounds__(kB) k_fmm_eval(FmmDevT<T2> f, Geo g, double* __restrict__ partial, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);  // [nd][p]
  // near-field sources of the 3 x 3 leaves, staged in rounds
  __shared__ float4 spa[kNearChunk];  // FP32: (x_hi, y_hi, x_lo, y_lo); float-float: (xh, xm, yh, ym)
  __shared__ float2 spb[NEARP == 2 ? kNearChunk : 1];  // float-float: (xl, yl)
  __shared__ float4 sq[kNearChunk];   // FP32: (q1, q2, -, -); float-float: (q1h, q1l, q2h, q2l)
  __shared__ __align__(16) int sid[kNearChunk];
  __shared__ int lst[10], lbeg[9];
  __shared__ float cen[6];  // FP32 instance: split leaf centre, 1/s, s
  const int b = blockIdx.x, bx = b % f.nb, by = b / f.nb;
  const int s0 = f.start[b], n = f.start[b + 1] - s0;
  if (n == 0) return;
  const long long box = lev_off(f.L) + b;
  if constexpr (NEARP == 2) {
    // float-float residuals: the local expansion split into hi + lo pairs
    float4* smf = reinterpret_cast<float4*>(smraw);
    for (int e = threadIdx.x; e < f.nd * f.p; e += kB) {
      const double2 a = f.lc[box * f.nd * f.p + e];
      const float rh = (float)a.x, ih = (float)a.y;
      smf[e] = make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
    }
  } else {
    for (int e = threadIdx.x; e < f.nd * f.p; e += kB) sm[e] = f.lc[box * f.nd * f.p + e];
  }
  const int y0 = max(0, by - 1), y1 = min(f.nb - 1, by + 1);
  const int x0 = max(0, bx - 1), x1 = min(f.nb - 1, bx + 1);
  if constexpr (NEARP == 1) leaf_center32(f, b, cen);
  if (threadIdx.x == 0) {
    int c = 0, tot = 0;
    for (int ny = y0; ny <= y1; ++ny)
      for (int nx = x0; nx <= x1; ++nx) {
        const int nl = ny * f.nb + nx;
        lbeg[c] = f.start[nl];
        lst[c] = tot;
        tot += f.start[nl + 1] - f.start[nl];
        ++c;
      }
    for (int k = c; k < 10; ++k) lst[k] = tot;
  }
  __syncthreads();
  const int total = lst[9];
  double s;
  const double2 c = box_center(f, f.L, bx, by, s);
  const double inv_s = ldexp(f.Dinv, f.L);
  for (int j0 = 0; j0 < n; j0 += kB) {
    const int j = j0 + threadIdx.x;
    const bool act = j < n;
    const int i = act ? f.perm[s0 + j] : 0;
    double ox = 0.0, oy = 0.0;
    float oxf = 0.f, oyf = 0.f;  // FP32 instance
    const double nx1 = (NEARP != 1 && act) ? g.nx[i] : 0.0, ny1 = (NEARP != 1 && act) ? g.ny[i] : 0.0;
    if (NEARP == 2 && act) {
      // the far field in float-float on the FP32 pipe (Horner for F and F',
      // then the kernel's combination), about the leaf centre
      const float4* smf = reinterpret_cast<const float4*>(smraw);
      const double ux = (g.x[i] - c.x) * inv_s, uy = (g.y[i] - c.y) * inv_s;
      const cff U = cff_split(ux, uy);
      const float ish = (float)inv_s, isl = (float)(inv_s - (double)ish);
      cff F[3], dF[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (d < f.nd) {
          cff h = cff_load(smf[d * f.p + f.p - 1]), dh = cff_zero();
          for (int l = f.p - 2; l >= 0; --l) {
            dh = cff_fma(h, dh, U);                         // h + dh u (the old h)
            h = cff_fma(cff_load(smf[d * f.p + l]), h, U);  // a_l + h u
          }
          F[d] = h;
          dF[d] = cff_scale(dh, ish, isl);
        }
      }
      if (f.nd == 1) {
        const double2 f0 = cff_to(F[0]);
        ox = nx1 * f0.x - ny1 * f0.y;
      } else {
        const cff nu = cff_split(nx1, ny1), nub = cff_conj(nu);
        const float slh = (float)s, sll = (float)(s - (double)slh);
        // S3 = -F'_{q conj(z_j - c)} with c the leaf centre (channel cm holds that density / s)
        const cff S2 = cff_neg(dF[0]), S3 = cff_neg(cff_scale(dF[2], slh, sll));
        const cff S1 = F[0], S6 = F[1];
        const cff zb = cff_split(g.x[i] - c.x, -(g.y[i] - c.y));
        const cff w = cff_fma(cff_neg(S3), zb, S2);  // conj(z - c) S2 - S3
        cff tt = cff_zero();
        tt = cff_fma(tt, nub, cff_conj(w));
        tt = cff_fma(tt, nu, cff_conj(S1));
        tt = cff_fma(tt, nub, cff_conj(S6));
        tt = cff_fma(tt, nu, S1);
        const double2 t2 = cff_to(tt);
        ox = 0.25 * t2.x;
        oy = 0.25 * t2.y;
      }
    }
    if constexpr (NEARP == 1) {
      if (act) {
        // FP32 throughout: u from the hi/lo split of z and the block's split
        // centre (no FP64 instruction per target)
        const float4 P = g.pf[i];
        const float2 nn = g.nf[i];
        const float dxc = (P.x - cen[0]) + (P.z - cen[2]), dyc = (P.y - cen[1]) + (P.w - cen[3]);
        const float2 u = make_float2(dxc * cen[4], dyc * cen[4]);
        float2 F[3], dF[3];  // nd = 1 or 3 (operator channels), unrolled: registers
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (d < f.nd) {
            float2 h = sm[d * f.p + f.p - 1], dh = make_float2(0.f, 0.f);
            for (int l = f.p - 2; l >= 0; --l) {
              dh = cadd(cmul(dh, u), h);
              h = cadd(cmul(h, u), sm[d * f.p + l]);
            }
            F[d] = h;
            dF[d] = make_float2(dh.x * cen[4], dh.y * cen[4]);
          }
        }
        if (f.nd == 1) {
          oxf = nn.x * F[0].x - nn.y * F[0].y;
        } else {
          // the kernel's combination about the leaf centre, as in the FP64 instance
          const float2 nu = nn, nub = make_float2(nn.x, -nn.y);
          const float2 S2 = make_float2(-dF[0].x, -dF[0].y);
          const float2 S3 = make_float2(-cen[5] * dF[2].x, -cen[5] * dF[2].y);
          const float2 S1 = F[0], S6 = F[1];
          float2 w = cmul(make_float2(dxc, -dyc), S2);
          w.x -= S3.x;
          w.y -= S3.y;
          float2 tt = cmul(nub, cconj(w));
          tt = cadd(tt, cmul(nu, cconj(S1)));
          tt = cadd(tt, cmul(nub, cconj(S6)));
          tt = cadd(tt, cmul(nu, S1));
          oxf = 0.25f * tt.x;
          oyf = 0.25f * tt.y;
        }
      }
    }
    if (NEARP == 0 && act) {
      const double2 zi = make_double2(g.x[i], g.y[i]);
      const T2 u = cx<T2>((zi.x - c.x) * inv_s, (zi.y - c.y) * inv_s);
      using R = decltype(u.x);
      const R is = (R)inv_s;
      T2 F[kMaxNd], dF[kMaxNd];
      for (int d = 0; d < f.nd; ++d) {
        // Horner for F and F' in u
        T2 h = sm[d * f.p + f.p - 1], dh = cx<T2>(0.0, 0.0);
        for (int l = f.p - 2; l >= 0; --l) {
          dh = cadd(cmul(dh, u), h);
          h = cadd(cmul(h, u), sm[d * f.p + l]);
        }
        F[d] = h;
        dF[d] = h;
        dF[d].x = dh.x * is;
        dF[d].y = dh.y * is;
      }
      if constexpr (NEARP == 0) {
        // near field: 3 x 3 leaves, as Cauchy terms
        for (int ny = y0; ny <= y1; ++ny) {
          for (int nx = x0; nx <= x1; ++nx) {
            const int nl = ny * f.nb + nx;
            for (int k = f.start[nl]; k < f.start[nl + 1]; ++k) {
              const int i2 = f.perm[k];
              if (i2 == i) continue;
              const double rx = zi.x - g.x[i2], ry = zi.y - g.y[i2];
              const double inv = 1.0 / (rx * rx + ry * ry);
              const double2 r1 = make_double2(rx * inv, -ry * inv);  // 1/(z_i - z_j)
              const double2 r2 = cmul(r1, r1);
              for (int d = 0; d < f.nd; ++d) {
                double2 q = f.Q[(long long)i2 * f.nd + (d == f.cm ? 0 : d)];
                if (d == f.cm)  // leaf-relative moment density q conj(z_j - c)/s
                  q = cmul(q, make_double2((g.x[i2] - c.x) * inv_s, -(g.y[i2] - c.y) * inv_s));
                cfma(F[d], q, r1);
                cfma(dF[d], make_double2(-q.x, -q.y), r2);
              }
            }
          }
        }
      }
      // the kernel's combination of the Cauchy sums, in the expansions' precision
      // (about the leaf centre its terms do not cancel)
      if (f.nd == 1) {
        ox = (double)((R)nx1 * F[0].x - (R)ny1 * F[0].y);
      } else {
        const T2 nu = cx<T2>(nx1, ny1), nub = cx<T2>(nx1, -ny1);
        const R sl = (R)s;
        // S3 = -F'_{q conj(z_j - c)} with c the leaf centre (channel cm holds that density / s)
        T2 S2 = dF[0], S3 = dF[2];
        S2.x = -S2.x;
        S2.y = -S2.y;
        S3.x = -sl * S3.x;
        S3.y = -sl * S3.y;
        const T2 S1 = F[0], S6 = F[1];
        const T2 zb = cx<T2>(zi.x - c.x, -(zi.y - c.y));
        T2 w = cmul(zb, S2);
        w.x -= S3.x;
        w.y -= S3.y;
        T2 tt = cmul(nub, cconj(w));
        tt = cadd(tt, cmul(nu, cconj(S1)));
        tt = cadd(tt, cmul(nub, cconj(S6)));
        tt = cadd(tt, cmul(nu, S1));
        ox = 0.25 * (double)tt.x;
        oy = 0.25 * (double)tt.y;
      }
    }
    if constexpr (NEARP != 0) {
      // near field as the real kernel, sources staged through shared memory
      float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 tn = make_float2(0.f, 0.f);
      FFTarget t;
      if (act) {
        if (NEARP == 1) {
          tp = g.pf[i];
          tn = g.nf[i];
        } else {
          const float4 pp = g.xff[i];
          const float2 pl = g.xfl[i];
          t.xh = pp.x;
          t.xm = pp.y;
          t.yh = pp.z;
          t.ym = pp.w;
          t.xl = pl.x;
          t.yl = pl.y;
          t.n = g.nff[i];
        }
      }
      float ax = 0.f, ay = 0.f, axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f;
      if constexpr (NEARP == 1) {
        // FP32: two sources a packed FP32x2 operation, staged in pairs
        // (positions hi and lo, strengths, node ids); an odd count is padded
        // with a zero-strength source far from everything
        float4* sp2 = spa;                  // [kNearChunk / 2] (xh0, xh1, yh0, yh1)
        float4* sl2 = spa + kNearChunk / 2;  // [kNearChunk / 2] (xl0, xl1, yl0, yl1)
        float4* sq2 = sq;                   // [kNearChunk / 2] (q1_0, q1_1, q2_0, q2_1)
        int2* sid2 = reinterpret_cast<int2*>(sid);
        const float2 TXH = make_float2(tp.x, tp.x), TYH = make_float2(tp.y, tp.y);
        const float2 TXL = make_float2(tp.z, tp.z), TYL = make_float2(tp.w, tp.w);
        const float2 NX = make_float2(tn.x, tn.x), NY = make_float2(tn.y, tn.y);
        float2 AX = make_float2(0.f, 0.f), AY = AX;
        for (int v0 = 0; v0 < total; v0 += kNearChunk) {
          const int m = min(kNearChunk, total - v0), m2 = (m + 1) >> 1;
          __syncthreads();
          for (int e2 = threadIdx.x; e2 < m2; e2 += kB) {
            float4 P[2];
            float2 q[2];
            int id[2];
            for (int h = 0; h < 2; ++h) {
              const int e = 2 * e2 + h;
              P[h] = make_float4(1e15f, 1e15f, 0.f, 0.f);
              q[h] = make_float2(0.f, 0.f);
              id[h] = -1;
              if (e < m) {
                const int vv = v0 + e;
                int lf = 0;
                while (vv >= lst[lf + 1]) ++lf;
                const int i2 = f.perm[lbeg[lf] + (vv - lst[lf])];
                P[h] = g.pf[i2];
                q[h] = f.Qf[i2];
                id[h] = i2;
              }
            }
            sp2[e2] = make_float4(P[0].x, P[1].x, P[0].y, P[1].y);
            sl2[e2] = make_float4(P[0].z, P[1].z, P[0].w, P[1].w);
            sq2[e2] = make_float4(q[0].x, q[1].x, q[0].y, q[1].y);
            sid2[e2] = make_int2(id[0], id[1]);
          }
          __syncthreads();
          if (act) {
            for (int e2 = 0; e2 < m2; ++e2) {
              const float4 P = sp2[e2], PL = sl2[e2], Q = sq2[e2];
              const int2 S = sid2[e2];
              // exact leading differences, as the scalar pair
              const float2 dx = __fadd2_rn(__fadd2_rn(TXH, make_float2(-P.x, -P.y)),
                                           __fadd2_rn(TXL, make_float2(-PL.x, -PL.y)));
              const float2 dy = __fadd2_rn(__fadd2_rn(TYH, make_float2(-P.z, -P.w)),
                                           __fadd2_rn(TYL, make_float2(-PL.z, -PL.w)));
              const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
              const float2 inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
              float2 cc;
              if (f.nd == 1) {
                cc = __fmul2_rn(make_float2(Q.x, Q.y), inv);
              } else {
                const float2 rq = __ffma2_rn(dx, make_float2(Q.x, Q.y), __fmul2_rn(dy, make_float2(Q.z, Q.w)));
                const float2 rn = __ffma2_rn(dx, NX, __fmul2_rn(dy, NY));
                cc = __fmul2_rn(__fmul2_rn(rq, rn), __fmul2_rn(inv, inv));
              }
              float2 cx2 = __fmul2_rn(cc, dx), cy2 = __fmul2_rn(cc, dy);
              if (S.x == i) cx2.x = cy2.x = 0.f;  // the self pair (r = 0)
              if (S.y == i) cx2.y = cy2.y = 0.f;
              AX = __fadd2_rn(AX, cx2);
              AY = __fadd2_rn(AY, cy2);
            }
          }
        }
        ax = AX.x + AX.y;
        ay = AY.x + AY.y;
      } else {
        // float-float: one source at a time, float-float sums
        for (int v0 = 0; v0 < total; v0 += kNearChunk) {
          const int m = min(kNearChunk, total - v0);
          __syncthreads();
          for (int e = threadIdx.x; e < m; e += kB) {
            const int vv = v0 + e;
            int lf = 0;
            while (vv >= lst[lf + 1]) ++lf;
            const int i2 = f.perm[lbeg[lf] + (vv - lst[lf])];
            sid[e] = i2;
            const double2 q = f.Q[(long long)i2 * f.nd];
            spa[e] = g.xff[i2];
            spb[e] = g.xfl[i2];
            const float q1h = (float)q.x, q2h = (float)q.y;
            sq[e] = make_float4(q1h, (float)(q.x - (double)q1h), q2h, (float)(q.y - (double)q2h));
          }
          __syncthreads();
          if (act) {
            for (int e = 0; e < m; ++e) {
              if (sid[e] == i) continue;
              float cxh, cxl, cyh, cyl;
              if (f.nd == 1)
                ff_pair<0>(t, spa[e], spb[e], sq[e], cxh, cxl, cyh, cyl);
              else
                ff_pair<1>(t, spa[e], spb[e], sq[e], cxh, cxl, cyh, cyl);
              ff_acc(axh, axl, cxh, cxl);
              ff_acc(ayh, ayl, cyh, cyl);
            }
          }
        }
      }
      if (NEARP == 2) {
        ax = 0.f;  // unused
        const double dax = (double)axh + (double)axl, day = (double)ayh + (double)ayl;
        if (f.nd == 1)
          ox += nx1 * dax + ny1 * day;
        else {
          ox += dax;
          oy += day;
        }
      } else {
        if (f.nd == 1) {
          oxf += tn.x * ax + tn.y * ay;
        } else {
          oxf += ax;
          oyf += ay;
        }
        ox = (double)oxf;
        oy = (double)oyf;
      }
    }
    if (act) {
      if (f.nd == 1) {
        partial[i] = ox;
      } else {
        partial[2 * i] = ox;
        partial[2 * i + 1] = oy;
      }
    }
  }
}

// Output densities at the boundary nodes (v = sqrt(w)-scaled total density):
// Laplace channel 0 = q = w nu (logarithm); Stokes f = w (nu1 + i nu2):
// channels f1, f2 (logarithm), f and f conj(z - c0) (Cauchy).
__global__ void k_fmm_out_density(Geo g, int nd, double cx0, double cy0, const double* __restrict__ v, double2* Q) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.M; i += gridDim.x * blockDim.x) {
    if (nd == 1) {
      Q[i] = make_double2(g.sw[i] * v[i], 0.0);
    } else {
      const double2 fq = make_double2(g.sw[i] * v[2 * i], g.sw[i] * v[2 * i + 1]);
      Q[4 * i] = make_double2(fq.x, 0.0);
      Q[4 * i + 1] = make_double2(fq.y, 0.0);
      Q[4 * i + 2] = fq;
      Q[4 * i + 3] = cmul(fq, make_double2(g.x[i] - cx0, -(g.y[i] - cy0)));
    }
  }
}

// Output targets: z0 per body (Laplace) or z0, z0 + delta e1, z0 + delta e2
// (Stokes); their leaves and the target counts of the leaves.
__global__ void k_fmm_targets(Geo g, int per, int L, double x0, double y0, double D, double* tx, double* ty,
                              int* tleaf, int* tcount_leaf) {
  const int T = g.N * per, nb = 1 << L;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    const int i = t / per, k = t % per;
    const double d = g.delta[i];
    const double x = g.zx[i] + (k == 1 ? d : 0.0), y = g.zy[i] + (k == 2 ? d : 0.0);
    tx[t] = x;
    ty[t] = y;
    int ix = (int)((x - x0) / D * nb), iy = (int)((y - y0) / D * nb);
    ix = min(max(ix, 0), nb - 1);
    iy = min(max(iy, 0), nb - 1);
    tleaf[t] = iy * nb + ix;
    atomicAdd(&tcount_leaf[iy * nb + ix], 1);
  }
}

// Single layers at the output targets: local expansion plus the 3 x 3 near
// leaves, in the layout of the direct output sums (Laplace: sum w nu log r^2;
// Stokes: sum [-log|r| f + r (r . f)/|r|^2] as a 2-vector).
constexpr int kTW = 8;  // targets (one warp each) per block of k_fmm_eval_targets

// One warp per target: the lanes split the near-field sources of the 3 x 3
// leaves (one reciprocal and one table-driven logarithm a pair), their sums
// are reduced across the warp in a fixed order, and lane 0 adds the local
// expansions of the target's leaf (Horner) and writes the output.
__global__ void __launch_bounds__(32 * kTW) k_fmm_eval_targets(FmmDev f, Geo g, int kind, int T,
                                                            const double* __restrict__ tx,
                                                            const double* __restrict__ ty,
                                                            const int* __restrict__ tleaf, double c0x, double c0y,
                                                            double* __restrict__ part) {
  __shared__ double2 ltab[kLogTab];
  log_table_fill(ltab);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int t = blockIdx.x * kTW + (threadIdx.x >> 5);
  if (t >= T) return;
  const int b = tleaf[t], bx = b % f.nb, by = b / f.nb;
  const long long box = lev_off(f.L) + b;
  const double x = tx[t], y = ty[t];
  double2 val[kMaxNd];
  for (int d = 0; d < kMaxNd; ++d) val[d] = make_double2(0.0, 0.0);
  for (int ny = max(0, by - 1); ny <= min(f.nb - 1, by + 1); ++ny)
    for (int nx = max(0, bx - 1); nx <= min(f.nb - 1, bx + 1); ++nx) {
      const int nl = ny * f.nb + nx;
      for (int k = f.start[nl] + lane; k < f.start[nl + 1]; k += 32) {
        const int j = f.perm[k];
        const double rx = x - g.x[j], ry = y - g.y[j];
        const double r2 = rx * rx + ry * ry;
        const double lg = 0.5 * log_tab(r2, ltab);
        for (int d = 0; d < f.nlog; ++d) val[d].x += f.Q[(long long)j * f.nd + d].x * lg;
        const double ir2 = 1.0 / r2;
        const double2 inv = make_double2(rx * ir2, -ry * ir2);
        for (int d = f.nlog; d < f.nd; ++d) cfma(val[d], f.Q[(long long)j * f.nd + d], inv);
      }
    }
  for (int d = 0; d < f.nd; ++d) {
    val[d].x = warp_sum(val[d].x);
    val[d].y = warp_sum(val[d].y);
  }
  if (lane != 0) return;
  double s;
  const double2 c = box_center(f, f.L, bx, by, s);
  const double2 u = make_double2((x - c.x) / s, (y - c.y) / s);
  for (int d = 0; d < f.nd; ++d) {
    const double2* lc = f.lc + (box * f.nd + d) * f.p;
    double2 h = lc[f.p - 1];
    for (int l = f.p - 2; l >= 0; --l) h = cadd(cmul(h, u), lc[l]);
    val[d] = cadd(h, val[d]);
  }
  if (kind == 0) {
    part[t] = 2.0 * val[0].x;
  } else {
    double2 ftot = make_double2(0.0, 0.0);  // sum of f over all nodes: the level-2 moments a_0
    for (int q = 0; q < 16; ++q) {
      const long long b2 = lev_off(2) + q;
      if (f.count[b2] > 0) ftot = cadd(ftot, f.mp[(b2 * f.nd + 2) * f.p]);
    }
    double2 w = cmul(make_double2(x - c0x, -(y - c0y)), val[2]);
    w = make_double2(w.x - val[3].x, -(w.y - val[3].y));  // conj(conj(t - c0) F_f - F_{f conj(z - c0)})
    part[2 * t] = -val[0].x + 0.5 * ftot.x + 0.5 * w.x;
    part[2 * t + 1] = -val[1].x + 0.5 * ftot.y + 0.5 * w.y;
  }
}

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// Translation operators for order p in the layout of tab_alpha..tab_size.
std::vector<std::complex<double>> build_ops(int p) {
  using C = std::complex<double>;
  std::vector<double> bin((2 * p + 1) * (2 * p + 1), 0.0);
  auto B = [&](int a, int b) -> double& { return bin[a * (2 * p + 1) + b]; };
  for (int a = 0; a <= 2 * p; ++a) {
    B(a, 0) = 1.0;
    for (int b = 1; b <= a; ++b) B(a, b) = B(a - 1, b - 1) + (b <= a - 1 ? B(a - 1, b) : 0.0);
  }
  std::vector<C> ops((size_t)tab_size(p), C(0, 0));
  auto at = [&](int o, int in, int out) -> C& { return ops[((size_t)o * p + in) * p + out]; };
  for (int c = 0; c < 4; ++c) {
    const C w(((c & 1) - 0.5) / 2.0, ((c >> 1) - 0.5) / 2.0);
    for (int k = 0; k < p; ++k)
      for (int m = 0; m <= k; ++m) at(c, m, k) = B(k, m) * std::pow(0.5, m) * std::pow(w, k - m);  // M2M
    for (int m = 0; m < p; ++m)
      for (int l = m; l < p; ++l) at(4 + c, l, m) = B(l, m) * std::pow(0.5, m) * std::pow(w, l - m);  // L2L
  }
  // M2L factors.  Cauchy: (d + u)^-(k+1) = sum_l C(k+l, l) (-1)^l u^l d^-(k+l+1).
  // Logarithm: log(d + u) = log d + sum_l (-1)^(l+1) (u/d)^l / l and
  // (d + u)^-k = sum_l C(k+l-1, l) (-1)^l u^l d^-(k+l); the log s part of log d
  // is added by the kernel.
  const size_t A = tab_alpha(p), Bt = tab_beta(p), G = tab_gamma(p), P = tab_pascal(p);
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      if (std::abs(dx) <= 1 && std::abs(dy) <= 1) continue;
      const size_t o = (size_t)(dx + 3) + 7 * (dy + 3);
      const C Dinv = 1.0 / C(dx, dy);
      for (int k = 0; k < p; ++k) {
        ops[A + o * p + k] = std::pow(Dinv, k);
        ops[A + (kOffs + o) * p + k] = k == 0 ? C(0, 0) : std::pow(Dinv, k) / (double)k;
      }
      for (int l = 0; l < p; ++l) {
        const double sg = (l & 1) ? -1.0 : 1.0;
        ops[Bt + o * p + l] = sg * std::pow(Dinv, l + 1);
        ops[Bt + (kOffs + o) * p + l] = -sg * std::pow(Dinv, l);
        ops[G + o * p + l] = l == 0 ? std::log(C(dx, dy)) : -sg * std::pow(Dinv, l) / (double)l;
      }
    }
  for (int k = 0; k < p; ++k)
    for (int l = 0; l < p; ++l) {
      ops[P + (size_t)k * p + l] = B(k + l, l);
      ops[P + ((size_t)p + k) * p + l] = k == 0 ? 0.0 : B(k + l - 1, l);
    }
  return ops;
}

}  // namespace

struct FmmState {
  int L = 0, nb = 0, nleaf = 0, kind = 0, M = 0, N = 0;
  double x0 = 0, y0 = 0, D = 0;
  long long nbox = 0;
  // device buffers (stream-ordered), grown on demand
  char* buf = nullptr;
  size_t buf_size = 0;
  int *leaf = nullptr, *perm = nullptr, *tmp = nullptr, *start = nullptr, *cursor = nullptr, *count = nullptr;
  int *tcount = nullptr, *tleaf = nullptr;
  double *tx = nullptr, *ty = nullptr;
  double2 *Q = nullptr, *mp = nullptr, *lc = nullptr;
  float4* cen32 = nullptr;  // per leaf: centre split as float hi + lo (x_h, y_h, x_l, y_l)
  double* scal = nullptr;
  int pmax = 0;
  // operators per order (FP64, and their FP32 copies)
  std::vector<std::pair<int, double2*>> ops;
  std::vector<std::pair<int, float2*>> ops32;
  // float-float M2L: split multipoles and the split factor tables per order
  float4* mpff = nullptr;
  std::vector<std::pair<int, float*>> opsff;
};

void fmm_free(FmmState* f, cudaStream_t s) {
  if (!f) return;
  if (f->buf) cudaFreeAsync(f->buf, s);
  for (auto& o : f->ops) cudaFreeAsync(o.second, s);
  for (auto& o : f->ops32) cudaFreeAsync(o.second, s);
  for (auto& o : f->opsff) cudaFreeAsync(o.second, s);
  delete f;
}

// Build the tree for the staged geometry (one host round trip for the box).
int fmm_setup(FmmState*& f, const Geo& g, int kind, const int* orders, int norders, cudaStream_t s,
              std::string& err, int leaf_nodes) {
  if (leaf_nodes <= 0) leaf_nodes = kDefaultLeafNodes;
  int pmax = 0;
  for (int k = 0; k < norders; ++k) {
    if (orders[k] < 2 || orders[k] > kMaxP) {
      err = "FMM order must be in 2.." + std::to_string(kMaxP);
      return BIE_ERR_INVALID;
    }
    pmax = std::max(pmax, orders[k]);
  }
  if (!f) f = new FmmState();
  auto ck = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess) err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaSuccess;
  };
  // bounding square and total length
  double* scal = nullptr;
  if (!f->scal) {
    if (!ck(cudaMallocAsync(reinterpret_cast<void**>(&f->scal), 4 * sizeof(double), s), "fmm scal")) return BIE_ERR_CUDA;
  }
  scal = f->scal;
  k_fmm_box<<<1, kBoxT, 0, s>>>(g, scal);
  note_launches(1);
  double h[4];
  if (!ck(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s), "fmm box") ||
      !ck(cudaStreamSynchronize(s), "fmm box sync"))
    return BIE_ERR_CUDA;
  f->x0 = h[0];
  f->y0 = h[1];
  f->D = h[2];
  // leaf level: the finest level whose non-empty leaves hold at least
  // leaf_nodes nodes (default 24); nodes on curves of total length P occupy
  // about min(4^L, 1.3 P 2^L / D) leaves
  int L = 2;
  for (int l = 2; l <= 10; ++l) {
    const double boxes = fmin((double)(1LL << (2 * l)), 1.3 * h[3] * (double)(1 << l) / f->D);
    if ((double)g.M / fmax(boxes, 1.0) >= (double)leaf_nodes) L = l;
  }
  f->L = L;
  f->nb = 1 << L;
  f->nleaf = f->nb * f->nb;
  f->nbox = lev_off(L + 1);
  f->kind = kind;
  f->M = g.M;
  f->N = g.N;
  const int nd = kMaxNd;  // room for the output channels
  f->pmax = pmax;
  // buffers
  auto pad = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t need = 3 * pad((size_t)g.M * 4) + 2 * pad(((size_t)f->nleaf + 1) * 4) + 2 * pad((size_t)f->nbox * 4) +
                      pad((size_t)g.M * nd * 16) + 3 * pad((size_t)f->nbox * nd * pmax * 16) +
                      pad((size_t)3 * g.N * 4) + 2 * pad((size_t)3 * g.N * 8) + pad((size_t)f->nleaf * 16);
  if (need > f->buf_size) {
    if (f->buf) cudaFreeAsync(f->buf, s);
    f->buf = nullptr;
    f->buf_size = 0;
    if (!ck(cudaMallocAsync(reinterpret_cast<void**>(&f->buf), need, s), "fmm buffers")) return BIE_ERR_CUDA;
    f->buf_size = need;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = f->buf + off;
    off += pad(bytes);
    return p;
  };
  f->leaf = (int*)take((size_t)g.M * 4);
  f->perm = (int*)take((size_t)g.M * 4);
  f->tmp = (int*)take((size_t)g.M * 4);
  f->start = (int*)take(((size_t)f->nleaf + 1) * 4);
  f->cursor = (int*)take(((size_t)f->nleaf + 1) * 4);
  f->count = (int*)take((size_t)f->nbox * 4);
  f->tcount = (int*)take((size_t)f->nbox * 4);
  f->tleaf = (int*)take((size_t)3 * g.N * 4);
  f->tx = (double*)take((size_t)3 * g.N * 8);
  f->ty = (double*)take((size_t)3 * g.N * 8);
  f->Q = (double2*)take((size_t)g.M * nd * 16);
  f->mp = (double2*)take((size_t)f->nbox * nd * pmax * 16);
  f->lc = (double2*)take((size_t)f->nbox * nd * pmax * 16);
  f->mpff = (float4*)take((size_t)f->nbox * nd * pmax * 16);
  f->cen32 = (float4*)take((size_t)f->nleaf * 16);
  // counting sort of the nodes by leaf, node order inside a leaf
  if (!ck(cudaMemsetAsync(f->cursor, 0, ((size_t)f->nleaf + 1) * 4, s), "fmm memset")) return BIE_ERR_CUDA;
  k_fmm_leaf<<<grid_for(g.M), 256, 0, s>>>(g, L, f->x0, f->y0, f->D, f->leaf, f->cursor);
  k_fmm_scan<<<1, 1024, 0, s>>>(f->cursor, f->nleaf, f->start);
  cudaMemsetAsync(f->cursor, 0, ((size_t)f->nleaf + 1) * 4, s);
  k_fmm_scatter<<<grid_for(g.M), 256, 0, s>>>(g.M, f->leaf, f->start, f->cursor, f->tmp);
  k_fmm_order<<<f->nleaf, 128, 0, s>>>(f->start, f->tmp, f->perm);
  k_fmm_leaf_counts<<<grid_for(f->nleaf), 256, 0, s>>>(f->start, f->nleaf, f->count + lev_off(L));
  for (int l = L - 1; l >= 0; --l) k_fmm_parent_counts<<<grid_for(1LL << (2 * l)), 256, 0, s>>>(l, f->count);
  k_fmm_leaf_centers<<<grid_for(f->nleaf), 256, 0, s>>>(f->nb, f->x0, f->y0, ldexp(f->D, -L), f->cen32);
  note_launches(7 + L);
  if (!ck(cudaGetLastError(), "fmm setup")) return BIE_ERR_CUDA;
  // translation operators, built before any capture of the apply
  for (int k = 0; k < norders; ++k) {
    const int p = orders[k];
    bool have = false;
    for (auto& o : f->ops) have |= o.first == p;
    if (have) continue;
    const auto host = build_ops(p);
    std::vector<float2> host32(host.size());
    for (size_t e = 0; e < host.size(); ++e)
      host32[e] = make_float2((float)host[e].real(), (float)host[e].imag());
    double2* ops = nullptr;
    float2* ops32 = nullptr;
    if (!ck(cudaMallocAsync(reinterpret_cast<void**>(&ops), host.size() * sizeof(double2), s), "fmm ops") ||
        !ck(cudaMallocAsync(reinterpret_cast<void**>(&ops32), host32.size() * sizeof(float2), s), "fmm ops") ||
        !ck(cudaMemcpyAsync(ops, host.data(), host.size() * sizeof(double2), cudaMemcpyHostToDevice, s), "fmm ops") ||
        !ck(cudaMemcpyAsync(ops32, host32.data(), host32.size() * sizeof(float2), cudaMemcpyHostToDevice, s),
            "fmm ops") ||
        !ck(cudaStreamSynchronize(s), "fmm ops"))
      return BIE_ERR_CUDA;
    f->ops.push_back({p, ops});
    f->ops32.push_back({p, ops32});
    // float-float splits of the M2L factors and of the Pascal matrices
    std::vector<float> hff((size_t)fftab_floats(p));
    auto split = [](double x, float& h, float& l) {
      h = (float)x;
      l = (float)(x - (double)h);
    };
    const size_t tabs[3] = {(size_t)tab_alpha(p), (size_t)tab_beta(p), (size_t)tab_gamma(p)};
    for (int t = 0; t < 5; ++t)  // alpha (2 types), beta (2 types), gamma
      for (int e = 0; e < kOffs * p; ++e) {
        const auto v = host[tabs[t / 2] + (size_t)(t % 2) * kOffs * p + e];
        float* q = hff.data() + ((size_t)t * kOffs * p + e) * 4;
        split(v.real(), q[0], q[2]);
        split(v.imag(), q[1], q[3]);
      }
    for (int e = 0; e < 2 * p * p; ++e) {
      float* q = hff.data() + (size_t)20 * kOffs * p + 2 * (size_t)e;
      split(host[(size_t)tab_pascal(p) + e].real(), q[0], q[1]);
    }
    float* opsff = nullptr;
    if (!ck(cudaMallocAsync(reinterpret_cast<void**>(&opsff), hff.size() * sizeof(float), s), "fmm ops") ||
        !ck(cudaMemcpyAsync(opsff, hff.data(), hff.size() * sizeof(float), cudaMemcpyHostToDevice, s), "fmm ops") ||
        !ck(cudaStreamSynchronize(s), "fmm ops"))
      return BIE_ERR_CUDA;
    f->opsff.push_back({p, opsff});
  }
  return BIE_OK;
}

namespace {

template <class T2, int PM>
void m2l_launch_pm(const FmmDevT<T2>& d, int L, const int* stop, cudaStream_t s) {
  const size_t sm = m2l_smem<T2>(d.p, d.nd, d.nlog, PM);
  const int threads = std::max(64, std::min(256, (d.nd * d.p + 31) / 32 * 32));
  cudaFuncSetAttribute(k_fmm_m2l<T2, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_fmm_m2l<T2, PM><<<(int)(lev_off(L + 1) - lev_off(2)), threads, sm, s>>>(d, stop);
}

// FP32 expansions of order <= 32 hold their Pascal rows in registers.
template <class T2>
void launch_m2l(const FmmDevT<T2>& d, int L, const int* stop, cudaStream_t s) {
  if constexpr (std::is_same<T2, float2>::value) {
    if (d.p <= 12) return m2l_launch_pm<T2, 12>(d, L, stop, s);
    if (d.p <= 16) return m2l_launch_pm<T2, 16>(d, L, stop, s);
    if (d.p <= 20) return m2l_launch_pm<T2, 20>(d, L, stop, s);
    if (d.p <= 24) return m2l_launch_pm<T2, 24>(d, L, stop, s);
    if (d.p <= 32) return m2l_launch_pm<T2, 32>(d, L, stop, s);
  }
  m2l_launch_pm<T2, 0>(d, L, stop, s);
}

// Shared memory of the M2M and L2L blocks: one box's expansions and one
// p x p translation matrix (above the default 48 KB for FP64 at high order).
template <class T2>
size_t tree_smem(int nd, int p) {
  const size_t sm = ((size_t)nd * p + (size_t)p * p) * sizeof(T2);
  if (sm > 48 * 1024) {
    cudaFuncSetAttribute(k_fmm_m2m<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_fmm_l2l<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  return sm;
}

// The upward pass, M2L, downward pass and evaluation with expansions of type T2.
template <class T2, int NEARP>
void fmm_passes(const FmmDevT<T2>& d, FmmState* f, const Geo& g, double* partial, const int* stop, cudaStream_t s) {
  const int p = d.p, nd = d.nd;
  const size_t sm_exp = (size_t)nd * p * sizeof(T2);
  const size_t sm_p2m = ((size_t)p * (kChunk + 1) + (size_t)kChunk * nd) * sizeof(T2);
  if constexpr (std::is_same<T2, float2>::value)
    k_fmm_p2m32<<<f->nleaf, kB, sm_p2m, s>>>(d, g, stop);
  else if constexpr (NEARP == 2)
    k_fmm_p2m_ff<<<f->nleaf, kB, sm_p2m, s>>>(d, g, stop);  // float4 = double2 in size
  else
    k_fmm_p2m<T2><<<f->nleaf, kB, sm_p2m, s>>>(d, g, stop);
  const size_t sm_tree = tree_smem<T2>(nd, p);
  for (int l = f->L - 1; l >= 2; --l) k_fmm_m2m<T2><<<1 << (2 * l), kB, sm_tree, s>>>(d, l, stop);
  bool done = false;
  if constexpr (std::is_same<T2, double2>::value && NEARP == 2) {
    // the float-float residual operator: float-float M2L
    const float* tab = nullptr;
    for (auto& o : f->opsff)
      if (o.first == p) tab = o.second;
    if (tab) {
      const long long nmp = (lev_off(f->L + 1) - lev_off(2)) * nd * p;
      k_fmm_mp_ff<<<grid_for(nmp), 256, 0, s>>>(d.mp + lev_off(2) * nd * p, nmp, f->mpff + lev_off(2) * nd * p);
      const size_t sm = (size_t)kListPad * nd * p * sizeof(float4);
      cudaFuncSetAttribute(k_fmm_m2l_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      k_fmm_m2l_ff<<<(int)(lev_off(f->L + 1) - lev_off(2)), kBFF, sm, s>>>(d, f->mpff, tab, stop);
      done = true;
    }
  }
  if (!done) launch_m2l(d, f->L, stop, s);
  for (int l = 2; l < f->L; ++l) k_fmm_l2l<T2><<<1 << (2 * (l + 1)), kB, sm_tree, s>>>(d, l, stop);
  k_fmm_eval<T2, NEARP><<<f->nleaf, kB, sm_exp, s>>>(d, g, partial, stop);
}

}  // namespace

void fmm_signature(const FmmState* f, long long sig[2]) {
  if (!f) {
    sig[0] = sig[1] = 0;
    return;
  }
  unsigned long long h = 1469598103934665603ULL;  // FNV-1a over the fields
  auto mix = [&](unsigned long long v) {
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xff;
      h *= 1099511628211ULL;
    }
  };
  unsigned long long u;
  memcpy(&u, &f->x0, 8);
  mix(u);
  memcpy(&u, &f->y0, 8);
  mix(u);
  memcpy(&u, &f->D, 8);
  mix(u);
  mix((unsigned long long)f->L);
  mix((unsigned long long)f->buf_size);
  mix((unsigned long long)f->M);
  sig[0] = (long long)(uintptr_t)f->buf;
  sig[1] = (long long)h;
}

cudaError_t fmm_pair_sum(FmmState* f, const Geo& g, int kind, int p, VecRef v, const double* sscale,
                         double* partial, const int* stop, cudaStream_t s, int near_prec) {
  if (!f || p > f->pmax || kind != f->kind) return cudaErrorInvalidValue;
  double2* ops = nullptr;
  float2* ops32 = nullptr;
  for (auto& o : f->ops)
    if (o.first == p) ops = o.second;
  for (auto& o : f->ops32)
    if (o.first == p) ops32 = o.second;
  if (!ops || !ops32) return cudaErrorInvalidValue;  // fmm_setup prepares every order
  const int nd = kind == 0 ? 1 : 3;
  if (near_prec == 1) {
    // the inner solves' operator: FP32 strengths, expansions (in the FP64
    // buffers) and near field
    float2* Qf = reinterpret_cast<float2*>(f->Q);
    k_fmm_density32<<<grid_for(g.M), 256, 0, s>>>(g, nd, v, sscale, Qf, stop);
    FmmDevT<float2> d{f->L,     f->nb,     p,        nd,       g.M,     0,       kind == 1 ? 2 : -1,
                      f->x0,    f->y0,     f->D,     1.0 / f->D, f->leaf,  f->perm, f->start,
                      f->count, f->count,  f->Q,     reinterpret_cast<float2*>(f->mp),
                      reinterpret_cast<float2*>(f->lc), ops32};
    d.Qf = Qf;
    d.cen32 = f->cen32;
    d.is32 = (float)ldexp(1.0 / f->D, f->L);
    d.s32 = (float)ldexp(f->D, -f->L);
    fmm_passes<float2, 1>(d, f, g, partial, stop, s);
  } else {
    k_fmm_density<<<grid_for(g.M), 256, 0, s>>>(g, nd, f->x0 + 0.5 * f->D, f->y0 + 0.5 * f->D, v, sscale, f->Q,
                                                 stop);
    const FmmDev d{f->L,    f->nb,    p,     nd,    g.M,   0,   kind == 1 ? 2 : -1, f->x0, f->y0, f->D, 1.0 / f->D, f->leaf,
                   f->perm, f->start, f->count, f->count, f->Q, f->mp, f->lc,  ops};
    if (near_prec == 2)
      fmm_passes<double2, 2>(d, f, g, partial, stop, s);
    else
      fmm_passes<double2, 0>(d, f, g, partial, stop, s);
  }
  note_launches(4 + 2 * std::max(0, f->L - 2) + (near_prec == 2 ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace bie

namespace bie {

// The output single layers at the interior targets by the FMM of order p
// (logarithm and Cauchy channels on the source tree of fmm_setup).
cudaError_t fmm_output(FmmState* f, const Geo& g, int kind, int p, const double* v, double* part, cudaStream_t s,
                       bool ff) {
  if (!f || p > f->pmax || kind != f->kind) return cudaErrorInvalidValue;
  double2* ops = nullptr;
  for (auto& o : f->ops)
    if (o.first == p) ops = o.second;
  if (!ops) return cudaErrorInvalidValue;
  const int nd = kind == 0 ? 1 : 4, nlog = kind == 0 ? 1 : 2, per = kind == 0 ? 1 : 3;
  const int T = g.N * per;
  const double c0x = f->x0 + 0.5 * f->D, c0y = f->y0 + 0.5 * f->D;
  cudaError_t e = cudaMemsetAsync(f->tcount, 0, (size_t)f->nbox * 4, s);
  if (e != cudaSuccess) return e;
  k_fmm_targets<<<grid_for(T), 256, 0, s>>>(g, per, f->L, f->x0, f->y0, f->D, f->tx, f->ty, f->tleaf,
                                          f->tcount + lev_off(f->L));
  for (int l = f->L - 1; l >= 0; --l) k_fmm_parent_counts<<<grid_for(1LL << (2 * l)), 256, 0, s>>>(l, f->tcount);
  k_fmm_out_density<<<grid_for(g.M), 256, 0, s>>>(g, nd, c0x, c0y, v, f->Q);
  FmmDev d{f->L, f->nb, p, nd, g.M, nlog, -1, f->x0, f->y0, f->D, 1.0 / f->D, f->leaf, f->perm, f->start, f->count, f->tcount,
           f->Q, f->mp, f->lc, ops};
  const size_t sm_p2m = ((size_t)p * (kChunk + 1) + (size_t)kChunk * nd) * sizeof(double2);
  if (ff)
    k_fmm_p2m_ff<<<f->nleaf, kB, sm_p2m, s>>>(d, g, nullptr);  // float4 = double2 in size
  else
    k_fmm_p2m<double2><<<f->nleaf, kB, sm_p2m, s>>>(d, g, nullptr);
  const size_t sm_tree = tree_smem<double2>(nd, p);
  for (int l = f->L - 1; l >= 2; --l) k_fmm_m2m<double2><<<1 << (2 * l), kB, sm_tree, s>>>(d, l, nullptr);
  const float* tab = nullptr;
  for (auto& o : f->opsff)
    if (o.first == p) tab = o.second;
  if (ff && tab) {
    // float-float multipole-to-local step (the float-float refinement's solves)
    const long long nmp = (lev_off(f->L + 1) - lev_off(2)) * nd * p;
    k_fmm_mp_ff<<<grid_for(nmp), 256, 0, s>>>(f->mp + lev_off(2) * nd * p, nmp, f->mpff + lev_off(2) * nd * p);
    const size_t sm = (size_t)kListPad * nd * p * sizeof(float4);
    cudaFuncSetAttribute(k_fmm_m2l_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fmm_m2l_ff<<<(int)(lev_off(f->L + 1) - lev_off(2)), kBFF, sm, s>>>(d, f->mpff, tab, nullptr);
    note_launches(1);
  } else {
    launch_m2l(d, f->L, nullptr, s);
  }
  for (int l = 2; l < f->L; ++l) k_fmm_l2l<double2><<<1 << (2 * (l + 1)), kB, sm_tree, s>>>(d, l, nullptr);
  k_fmm_eval_targets<<<(T + kTW - 1) / kTW, 32 * kTW, 0, s>>>(d, g, kind, T, f->tx, f->ty, f->tleaf, c0x, c0y,
                                                               part);
  note_launches(7 + f->L + 2 * std::max(0, f->L - 2));
  return cudaGetLastError();
}

}  // namespace bie
