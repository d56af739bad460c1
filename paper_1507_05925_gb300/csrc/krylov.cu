// Device-resident restarted GMRES (FP64): classical Gram-Schmidt with one
// re-orthogonalisation pass (CGS2), Givens rotations, and a convergence flag in
// device memory so that a cycle runs without host round trips.  Every kernel
// returns at once when the flag is set, so the host may enqueue iterations
// ahead of the check.
//
// Grid reductions write per-block partials and the last block to finish (an
// atomic ticket) adds them in block order: results are deterministic.
#include <math.h>

#include "bie_internal.cuh"
#include "reduce.cuh"

namespace bie {

namespace {

constexpr int kBV = 256;
constexpr int kMaxBasis = 201;  // restart length <= 200

// Partial dot products of the thread's elements of w with V_0..V_{jc-1}; the
// per-block results land in part[blockIdx.x][i]; the last block reduces them
// into h[i] and returns true.
__device__ bool block_dots(const double* __restrict__ V, long long ld, const double* __restrict__ w,
                           long long n, int jc, double* __restrict__ part, double* __restrict__ h,
                           int* counter) {
  __shared__ double sh[kBV / 32][kMaxBasis];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * kBV;
  // four basis vectors per round: four independent load streams per thread
  int i = 0;
  for (; i + 4 <= jc; i += 4) {
    const double* __restrict__ V0 = V + (long long)i * ld;
    const double* __restrict__ V1 = V0 + ld;
    const double* __restrict__ V2 = V1 + ld;
    const double* __restrict__ V3 = V2 + ld;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
      const double wk = w[k];
      a0 += V0[k] * wk;
      a1 += V1[k] * wk;
      a2 += V2[k] * wk;
      a3 += V3[k] * wk;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
      a2 += __shfl_down_sync(0xffffffffu, a2, o);
      a3 += __shfl_down_sync(0xffffffffu, a3, o);
    }
    if (lane == 0) {
      sh[wid][i] = a0;
      sh[wid][i + 1] = a1;
      sh[wid][i + 2] = a2;
      sh[wid][i + 3] = a3;
    }
  }
  for (; i < jc; ++i) {
    const double* __restrict__ Vi = V + (long long)i * ld;
    double acc = 0.0;
    for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) acc += Vi[k] * w[k];
    acc = warp_sum(acc);
    if (lane == 0) sh[wid][i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < jc; i += kBV) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kBV / 32; ++q) s += sh[q][i];
    part[(long long)blockIdx.x * kMaxBasis + i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  for (int i = threadIdx.x; i < jc; i += kBV) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile double*)part)[(long long)b * kMaxBasis + i];
    h[i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

// sum_i c[i] V_i[k] for i < jc, four independent partial sums
__device__ __forceinline__ double combine(const double* __restrict__ V, long long ld, long long k,
                                          const double* c, int jc) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = 0;
  for (; i + 4 <= jc; i += 4) {
    s0 += c[i] * V[(long long)i * ld + k];
    s1 += c[i + 1] * V[(long long)(i + 1) * ld + k];
    s2 += c[i + 2] * V[(long long)(i + 2) * ld + k];
    s3 += c[i + 3] * V[(long long)(i + 3) * ld + k];
  }
  for (; i < jc; ++i) s0 += c[i] * V[(long long)i * ld + k];
  return (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(kBV) k_cgs_dots(const double* __restrict__ V, long long ld, VecRef wr,
                                                  long long n, KState* st, double* part, double* h1) {
  if (st->stop) return;
  block_dots(V, ld, wr.ptr(), n, st->j + 1, part, h1, &st->counter);
}

__global__ void __launch_bounds__(kBV) k_cgs_update_dots(const double* __restrict__ V, long long ld,
                                                         VecRef wr, long long n, KState* st, double* part,
                                                         const double* __restrict__ h1, double* h2) {
  if (st->stop) return;
  __shared__ double hs[kMaxBasis];
  const int jc = st->j + 1;
  for (int i = threadIdx.x; i < jc; i += kBV) hs[i] = h1[i];
  __syncthreads();
  double* __restrict__ w = wr.ptr();
  const long long stride = (long long)gridDim.x * kBV;
  for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
    w[k] = w[k] - combine(V, ld, k, hs, jc);
  }
  block_dots(V, ld, w, n, jc, part, h2, &st->counter);
}

// w -= V h2, ||w||, then (last block, one thread) the Hessenberg column j,
// the previous rotations, a new rotation and the residual estimate |g_{j+1}|.
__global__ void __launch_bounds__(kBV) k_cgs_update_norm(const double* __restrict__ V, long long ld,
                                                         VecRef wr, long long n, KState* st, double* part,
                                                         const double* __restrict__ h1,
                                                         const double* __restrict__ h2, double* H,
                                                         double* cs, double* sn, double* gv) {
  if (st->stop) return;
  __shared__ double hs[kMaxBasis];
  __shared__ double sh[kBV / 32];
  __shared__ int is_last;
  const int j = st->j;
  const int jc = j + 1;
  for (int i = threadIdx.x; i < jc; i += kBV) hs[i] = h2[i];
  __syncthreads();
  double* __restrict__ w = wr.ptr();
  const long long stride = (long long)gridDim.x * kBV;
  double nrm = 0.0;
  for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
    const double acc = w[k] - combine(V, ld, k, hs, jc);
    w[k] = acc;
    nrm += acc * acc;
  }
  nrm = block_sum<kBV>(nrm, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = nrm;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  double s = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile double*)part)[b];
  st->counter = 0;
  const int m = st->m;
  double* Hc = H + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = h1[i] + h2[i];
  const double hn = sqrt(s);
  Hc[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * Hc[i] + sn[i] * Hc[i + 1];
    Hc[i + 1] = -sn[i] * Hc[i] + cs[i] * Hc[i + 1];
    Hc[i] = t;
  }
  const double a = Hc[j], b = Hc[j + 1];
  const double r = hypot(a, b);
  const double c = r > 0.0 ? a / r : 1.0, sg = r > 0.0 ? b / r : 0.0;
  cs[j] = c;
  sn[j] = sg;
  Hc[j] = r;
  Hc[j + 1] = 0.0;
  gv[j + 1] = -sg * gv[j];
  gv[j] = c * gv[j];
  st->res = fabs(gv[j + 1]);
  st->hnext = hn;
  st->j = j + 1;
  st->iters += 1;
  if (st->res <= st->tol_abs || !(hn > 1e-300 * st->beta) || st->j >= m || st->iters >= st->maxit)
    st->stop = 1;
}

__global__ void k_normalize(VecRef wr, long long n, const KState* st) {
  if (st->stop) return;
  double* w = wr.ptr();
  const double inv = 1.0 / st->hnext;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    w[k] *= inv;
}

// Back substitution R y = g on the j x j triangle (single thread; j <= 200).
__global__ void k_triangular(const KState* st, const double* __restrict__ H, const double* __restrict__ gv,
                             double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int j = st->j, m = st->m;
  for (int i = j - 1; i >= 0; --i) {
    double s = gv[i];
    for (int k = i + 1; k < j; ++k) s -= H[(long long)k * (m + 1) + i] * y[k];
    y[i] = s / H[(long long)i * (m + 1) + i];
  }
}

__global__ void k_update_x(const double* __restrict__ V, long long ld, long long n, const KState* st,
                           const double* __restrict__ y, double* __restrict__ x) {
  __shared__ double ys[kMaxBasis];
  const int j = st->j;
  for (int i = threadIdx.x; i < j; i += blockDim.x) ys[i] = y[i];
  __syncthreads();
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    x[k] += combine(V, ld, k, ys, j);
  }
}

// r = f - y (y may be NULL: r = f), ||r|| into st->rnorm; with start_cycle the
// last block also opens a new cycle: g = (||r||, 0, ...), j = 0, stop if
// already below tolerance.
__global__ void __launch_bounds__(kBV) k_residual(const double* __restrict__ f, const double* __restrict__ y,
                                                  double* __restrict__ r, long long n, KState* st,
                                                  double* part, double* gv, int start_cycle) {
  __shared__ double sh[kBV / 32];
  __shared__ int is_last;
  double nrm = 0.0;
  const long long stride = (long long)gridDim.x * kBV;
  for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
    const double v = y ? f[k] - y[k] : f[k];
    r[k] = v;
    nrm += v * v;
  }
  nrm = block_sum<kBV>(nrm, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = nrm;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  double s = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile double*)part)[b];
  st->counter = 0;
  const double rn = sqrt(s);
  st->rnorm = rn;
  if (start_cycle) {
    if (st->pad[0]) {  // first call of a solve: tolerance relative to ||b||
      st->tol_abs = st->scratch[0] * rn;
      st->scratch[1] = rn;
      st->pad[0] = 0;
    }
    st->beta = rn;
    st->res = rn;
    st->j = 0;
    gv[0] = rn;
    st->stop = (rn <= st->tol_abs || st->iters >= st->maxit || !(rn > 0.0)) ? 1 : 0;
  }
}

__global__ void k_start_v0(const double* __restrict__ r, double* __restrict__ V0, long long n, const KState* st) {
  if (st->stop) return;
  const double inv = 1.0 / st->beta;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    V0[k] = r[k] * inv;
}

__global__ void k_axpy(double* __restrict__ x, const double* __restrict__ d, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    x[k] += d[k];
}

__global__ void k_fill0(double* __restrict__ x, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    x[k] = 0.0;
}

inline int elt_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

}  // namespace

int vec_grid(long long n) {
  long long b = (n + kBV - 1) / kBV;
  if (b > 608) b = 608;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t cgs_dots(const double* V, long long ld, VecRef w, long long n, KState* st, double* part,
                     double* h1, int grid, cudaStream_t s) {
  k_cgs_dots<<<grid, kBV, 0, s>>>(V, ld, w, n, st, part, h1);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t cgs_update_dots(const double* V, long long ld, VecRef w, long long n, KState* st,
                            double* part, const double* h1, double* h2, int grid, cudaStream_t s) {
  k_cgs_update_dots<<<grid, kBV, 0, s>>>(V, ld, w, n, st, part, h1, h2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t cgs_update_norm(const double* V, long long ld, VecRef w, long long n, KState* st,
                            double* part, const double* h1, const double* h2, double* H, double* cs,
                            double* sn, double* gv, int grid, cudaStream_t s) {
  k_cgs_update_norm<<<grid, kBV, 0, s>>>(V, ld, w, n, st, part, h1, h2, H, cs, sn, gv);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t normalize_next(VecRef w, long long n, KState* st, cudaStream_t s) {
  k_normalize<<<elt_grid(n), 256, 0, s>>>(w, n, st);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t gmres_update(const double* V, long long ld, long long n, KState* st, const double* H,
                         const double* gv, double* y, double* x, int grid, cudaStream_t s) {
  (void)grid;
  k_triangular<<<1, 32, 0, s>>>(st, H, gv, y);
  note_launches(1);
  k_update_x<<<elt_grid(n), 256, 0, s>>>(V, ld, n, st, y, x);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t residual_start(const double* f, const double* y, double* r, double* V0, long long n,
                           KState* st, double* part, double* gv, int start_cycle, int grid,
                           cudaStream_t s) {
  k_residual<<<grid, kBV, 0, s>>>(f, y, r, n, st, part, gv, start_cycle);
  note_launches(1);
  if (start_cycle) {
    k_start_v0<<<elt_grid(n), 256, 0, s>>>(r, V0, n, st);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t axpy(double* x, const double* d, long long n, cudaStream_t s) {
  k_axpy<<<elt_grid(n), 256, 0, s>>>(x, d, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t fill0(double* x, long long n, cudaStream_t s) {
  k_fill0<<<elt_grid(n), 256, 0, s>>>(x, n);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bie
