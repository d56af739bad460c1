// Device-resident restarted GMRES (FP64): classical Gram-Schmidt with one
// re-orthogonalisation pass (CGS2), Givens rotations, and a convergence flag in
// device memory so that a cycle runs without host round trips.  Every kernel
// returns at once when the flag is set, so the host may enqueue iterations
// ahead of the check.
//
// Grid reductions write per-block partials that are added in block order
// (by the last block to finish, through an atomic ticket, or by every block
// after a grid barrier): results are deterministic.
#include <math.h>

#include "bie_internal.cuh"
#include "reduce.cuh"

#include <algorithm>
#include <atomic>

namespace bie {

namespace {

constexpr int kBV = 256;
constexpr int kMaxBasis = 201;  // restart length <= 200

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

// ------------------------------------------------------------ fused Arnoldi
// One Arnoldi step after w = A z_j (w = V_{j+1}) in a single cooperative
// launch with three grid barriers: CGS2 (h1 = V^T w; w -= V h1; h2 = V^T w;
// w -= V h2), ||w||, the Hessenberg column with its Givens rotations and the
// residual estimate, v_{j+1} = w / ||w|| and, with the block-Jacobi
// preconditioner, z_{j+1} = P v_{j+1}.  After each barrier every CTA adds the
// per-CTA partials itself, in CTA order (deterministic; no atomics), so
// nothing else synchronises the grid.  In the last phase a CTA that owns a
// body reads that body's w, writes z and normalises v in place: every element
// is written only by its owner, after the owner has read it.

// Partial dot products of this CTA's elements of w with V_0..V_{jc-1} into
// out[0..jc).  NARROW (a grid of at most two CTAs per SM, few elements a
// CTA): warp u takes basis vectors u, u + 8, ..., its lanes stride the CTA's
// elements with two independent sums, one warp reduction per vector.  Wide
// grids: all threads take four vectors at a time, reduced through shared
// memory.  Both in a fixed order (deterministic).
template <bool NARROW>
__device__ __forceinline__ void arn_block_dots(const double* __restrict__ V, long long ld,
                                               const double* __restrict__ w, long long n, int jc,
                                               double* __restrict__ out, double (*sh)[kMaxBasis]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * kBV;
  if (NARROW) {
    const long long base = blockIdx.x * (long long)kBV;
    for (int i = wid; i < jc; i += kBV / 32) {
      const double* __restrict__ Vi = V + (long long)i * ld;
      double a0 = 0.0, a1 = 0.0;
      for (long long c = base; c < n; c += stride) {
#pragma unroll
        for (int u = 0; u < kBV / 32; u += 2) {
          const long long k0 = c + u * 32 + lane, k1 = k0 + 32;
          if (k0 < n) a0 = fma(Vi[k0], w[k0], a0);
          if (k1 < n) a1 = fma(Vi[k1], w[k1], a1);
        }
      }
      const double t = warp_sum(a0 + a1);
      if (lane == 0) out[i] = t;
    }
    __syncthreads();
    return;
  }
  int i = 0;
  for (; i + 4 <= jc; i += 4) {
    const double* __restrict__ V0 = V + (long long)i * ld;
    const double* __restrict__ V1 = V0 + ld;
    const double* __restrict__ V2 = V1 + ld;
    const double* __restrict__ V3 = V2 + ld;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
      const double wk = w[k];
      a0 = fma(V0[k], wk, a0);
      a1 = fma(V1[k], wk, a1);
      a2 = fma(V2[k], wk, a2);
      a3 = fma(V3[k], wk, a3);
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
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
    for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) acc = fma(Vi[k], w[k], acc);
    acc = warp_sum(acc);
    if (lane == 0) sh[wid][i] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < jc; q += kBV) {
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < kBV / 32; ++u) t += sh[u][q];
    out[q] = t;
  }
}

// Sum over CTAs b < gridDim.x of part[b * stride] (written by other CTAs
// before a barrier or ticket; read through L2), by one warp: lanes take
// b = lane, lane + 32, ... with independent loads, then a fixed-order warp
// reduction (deterministic).  The total is valid in lane 0.
__device__ __forceinline__ double warp_gather(const double* part, long long stride) {
  const int lane = threadIdx.x & 31;
  double t0 = 0.0, t1 = 0.0;
  int b = lane;
  for (; b + 32 < (int)gridDim.x; b += 64) {
    t0 += __ldcg(part + (long long)b * stride);
    t1 += __ldcg(part + (long long)(b + 32) * stride);
  }
  if (b < (int)gridDim.x) t0 += __ldcg(part + (long long)b * stride);
  return warp_sum(t0 + t1);
}

// hs[i] = sum over CTAs b of part[b][i], one warp per i.
__device__ __forceinline__ void arn_grid_sum(const double* part, int jc, double* hs) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < jc; i += kBV / 32) {
    const double t = warp_gather(part + i, kMaxBasis);
    if (lane == 0) hs[i] = t;
  }
  __syncthreads();
}

// Grid barrier for a cooperative launch (all CTAs co-resident): arrival
// counter plus generation number in the solver state.  The wait is bounded:
// after `spins` polls (about a second for the default) it records st->error,
// sets st->stop (so that every later kernel of the iteration returns at once)
// and gives up; a CTA that finds the error already recorded neither arrives
// nor waits.  Returns true when the barrier failed: the caller then returns,
// so a fault can never hang the GPU, and the host reports BIE_ERR_TIMEOUT.  The
// counter is left as it was; the next solve starts from a cleared state.
constexpr long long kBarrierSpins = 1LL << 24;

__device__ __forceinline__ bool grid_barrier(KState* st, long long spins) {
  __shared__ int failed;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* err = &st->error;
    int f = *err;
    if (!f) {
      volatile unsigned* gen = &st->bar_gen;
      const unsigned g0 = *gen;
      __threadfence();
      if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
        st->bar_count = 0;
        __threadfence();
        atomicAdd(&st->bar_gen, 1u);
      } else {
        long long it = 0;
        while (*gen == g0) {
          if (*err) {
            f = 1;
            break;
          }
          if (++it > spins) {
            atomicExch(&st->error, 1);
            atomicExch(&st->stop, 1);
            f = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    failed = f;
  }
  __syncthreads();
  return failed != 0;
}

// z = P v = 2 v + W v for one body's block-Jacobi block W (column-major
// nb x nb, FP16; off = its offset in the block array) and v = ws in shared
// memory, in FP32 arithmetic.  red8 holds 2 kBV float4.
__device__ __forceinline__ void bj_body_apply(const bj_t* __restrict__ B, long long off, int nb, const float* ws,
                                              double* __restrict__ z, float4* red8) {
  if ((nb & 7) == 0 && (off & 7) == 0 && (reinterpret_cast<uintptr_t>(z) & 15) == 0) {
    // 16-byte loads of eight consecutive rows: R row-octet slots (the
    // smallest power of two >= nb/8, from 8 to 64) x kBV/R column groups, so
    // that every thread streams part of the block (a body of 64 Stokes
    // nodes: 16 row octets x 16 groups of 8 columns, 8 loads in flight a
    // thread)
    const int no = nb >> 3;
    int R = 64;
    while (R > 8 && (R >> 1) >= no) R >>= 1;
    const int ng = kBV / R, qd = threadIdx.x & (R - 1), grp = threadIdx.x / R;
    const int per = (nb + ng - 1) / ng, cb = grp * per, ce = min(nb, cb + per);
    for (int q0 = 0; q0 < no; q0 += R) {
      const int q = q0 + qd;
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.f;
      if (q < no) {
        const uint4* __restrict__ Bq = reinterpret_cast<const uint4*>(B) + q;
#pragma unroll 4
        for (int col = cb; col < ce; ++col) {
          const uint4 b = Bq[(long long)col * no];
          const float x = ws[col];
          const __half2* h = reinterpret_cast<const __half2*>(&b);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float2 f = __half22float2(h[u]);
            acc[2 * u] = fmaf(f.x, x, acc[2 * u]);
            acc[2 * u + 1] = fmaf(f.y, x, acc[2 * u + 1]);
          }
        }
      }
      red8[2 * threadIdx.x] = make_float4(acc[0], acc[1], acc[2], acc[3]);
      red8[2 * threadIdx.x + 1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      __syncthreads();
      if (grp == 0 && q < no) {
        float4 t0 = red8[2 * qd], t1 = red8[2 * qd + 1];
        for (int u = 1; u < ng; ++u) {
          const float4 o0 = red8[2 * (u * R + qd)], o1 = red8[2 * (u * R + qd) + 1];
          t0 = make_float4(t0.x + o0.x, t0.y + o0.y, t0.z + o0.z, t0.w + o0.w);
          t1 = make_float4(t1.x + o1.x, t1.y + o1.y, t1.z + o1.z, t1.w + o1.w);
        }
        const float* v8 = ws + 8 * q;
        double2* zr = reinterpret_cast<double2*>(z + 8 * q);
        zr[0] = make_double2(fmaf(kBjShift, v8[0], t0.x), fmaf(kBjShift, v8[1], t0.y));
        zr[1] = make_double2(fmaf(kBjShift, v8[2], t0.z), fmaf(kBjShift, v8[3], t0.w));
        zr[2] = make_double2(fmaf(kBjShift, v8[4], t1.x), fmaf(kBjShift, v8[5], t1.y));
        zr[3] = make_double2(fmaf(kBjShift, v8[6], t1.z), fmaf(kBjShift, v8[7], t1.w));
      }
      __syncthreads();
    }
  } else {
    for (int r = threadIdx.x; r < nb; r += kBV) {
      float s0 = 0.f, s1 = 0.f;
      int col = 0;
#pragma unroll 4
      for (; col + 2 <= nb; col += 2) {
        s0 = fmaf(__half2float(B[(long long)col * nb + r]), ws[col], s0);
        s1 = fmaf(__half2float(B[(long long)(col + 1) * nb + r]), ws[col + 1], s1);
      }
      if (col < nb) s0 = fmaf(__half2float(B[(long long)col * nb + r]), ws[col], s0);
      z[r] = (double)fmaf(kBjShift, ws[r], s0 + s1);
    }
  }
}

// z = P v in FP64 arithmetic on the FP16 block (the FP64 GMRES: the
// preconditioner must be one fixed linear map to FP64 rounding, so that the
// Arnoldi relation A P V = V H holds to FP64 accuracy and x = P (V y) is the
// minimiser GMRES computed).
__device__ __forceinline__ void bj_body_apply64(const bj_t* __restrict__ B, int nb, const double* wd,
                                                double* __restrict__ z) {
  for (int r = threadIdx.x; r < nb; r += kBV) {
    double s0 = 0.0, s1 = 0.0;
    int col = 0;
#pragma unroll 4
    for (; col + 2 <= nb; col += 2) {
      s0 = fma((double)__half2float(B[(long long)col * nb + r]), wd[col], s0);
      s1 = fma((double)__half2float(B[(long long)(col + 1) * nb + r]), wd[col + 1], s1);
    }
    if (col < nb) s0 = fma((double)__half2float(B[(long long)col * nb + r]), wd[col], s0);
    z[r] = fma((double)kBjShift, wd[r], s0 + s1);
  }
}

// CTA 0, all threads: Hessenberg column j (hs1 + hs2, then ||w||), the
// previous rotations and the new one, the residual estimate and the stopping
// test.  The column and rotations are kept in shared memory (one thread
// applies the rotations; no global round trips in the chain).
__device__ __noinline__ void arn_hessenberg(const ArnoldiArgs& a, KState* st, int j, const double* hs1,
                                            const double* hs2, double hn) {
  // Hessenberg column j and the previous rotations in shared memory (one
  // thread applies the rotations; no global round trips in the chain)
  __shared__ double hcol[kMaxBasis + 1], css[kMaxBasis], sns[kMaxBasis];
  const int m = st->m;
  double* Hc = a.H + (long long)j * (m + 1);
  for (int i = threadIdx.x; i <= j; i += kBV) hcol[i] = hs1[i] + hs2[i];
  for (int i = threadIdx.x; i < j; i += kBV) {
    css[i] = a.cs[i];
    sns[i] = a.sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    hcol[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = css[i] * hcol[i] + sns[i] * hcol[i + 1];
      hcol[i + 1] = -sns[i] * hcol[i] + css[i] * hcol[i + 1];
      hcol[i] = t;
    }
    const double x = hcol[j], y = hcol[j + 1];
    const double r = hypot(x, y);
    const double c = r > 0.0 ? x / r : 1.0, sg = r > 0.0 ? y / r : 0.0;
    a.cs[j] = c;
    a.sn[j] = sg;
    hcol[j] = r;
    hcol[j + 1] = 0.0;
    const double g = a.gv[j];
    a.gv[j + 1] = -sg * g;
    a.gv[j] = c * g;
    st->res = fabs(sg * g);
    st->hnext = hn;
    st->j = j + 1;
    st->iters += 1;
    if (st->res <= st->tol_abs || !(hn > 1e-300 * st->beta) || st->j >= m || st->iters >= st->maxit)
      st->stop = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += kBV) Hc[i] = hcol[i];
}

template <bool NARROW>
__global__ void __launch_bounds__(kBV, NARROW ? 1 : 4) k_arnoldi(ArnoldiArgs a) {
  KState* st = a.st;
  if (st->stop) return;  // read by every CTA before the first barrier: uniform
  __shared__ double sh[kBV / 32][kMaxBasis];
  __shared__ double hs1[kMaxBasis], hs2[kMaxBasis];
  __shared__ double red[kBV / 32];
  __shared__ float ws[kBjMaxBlock];
  __shared__ double wsd[kBjMaxBlock];
  const int j = st->j, jc = j + 1;
  const long long n = a.n, ld = a.ld;
  double* __restrict__ w = a.V + (long long)(j + 1) * ld;
  const long long stride = (long long)gridDim.x * kBV;
  const long long G = gridDim.x;
  double* part1 = a.part;
  double* part2 = part1 + G * kMaxBasis;
  double* part3 = part2 + G * kMaxBasis;
  // h1 = V^T w
  arn_block_dots<NARROW>(a.V, ld, w, n, jc, part1 + blockIdx.x * kMaxBasis, sh);
  if ((int)blockIdx.x == a.fault_skip) return;  // test hook: this CTA never arrives
  if (grid_barrier(st, a.spins)) return;
  arn_grid_sum(part1, jc, hs1);
  // w -= V h1; h2 = V^T w
  for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride)
    w[k] = w[k] - combine(a.V, ld, k, hs1, jc);
  __syncthreads();
  arn_block_dots<NARROW>(a.V, ld, w, n, jc, part2 + blockIdx.x * kMaxBasis, sh);
  if (grid_barrier(st, a.spins)) return;
  arn_grid_sum(part2, jc, hs2);
  // w -= V h2; ||w||^2
  double nrm = 0.0;
  for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) {
    const double t = w[k] - combine(a.V, ld, k, hs2, jc);
    w[k] = t;
    nrm = fma(t, t, nrm);
  }
  nrm = block_sum<kBV>(nrm, red);
  if (threadIdx.x == 0) part3[blockIdx.x * kMaxBasis] = nrm;
  if (grid_barrier(st, a.spins)) return;
  __shared__ double hn_s;
  if (threadIdx.x < 32) {
    const double t = warp_gather(part3, kMaxBasis);
    if (threadIdx.x == 0) hn_s = sqrt(t);
  }
  __syncthreads();
  const double hn = hn_s;
  if (blockIdx.x == 0) arn_hessenberg(a, st, j, hs1, hs2, hn);
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  if (!a.blocks) {
    // v_{j+1} = w / ||w|| over this CTA's own elements
    for (long long k = blockIdx.x * (long long)kBV + threadIdx.x; k < n; k += stride) w[k] *= inv;
    return;
  }
  // per body: v = w inv (w read through L2: other CTAs wrote it), z = P v
  __shared__ float4 red4[2 * kBV];
  const int c = a.kind + 1;
  for (int i = blockIdx.x; i < a.g.N; i += (int)G) {
    const long long a0 = (long long)a.g.body_start[i] * c;
    const int nb = (a.g.body_start[i + 1] - a.g.body_start[i]) * c;
    if (nb > kBjMaxBlock) {
      for (int r = threadIdx.x; r < nb; r += kBV) {
        const double v = __ldcg(w + a0 + r) * inv;
        w[a0 + r] = v;
        a.z[a0 + r] = v;
      }
      continue;
    }
    for (int r = threadIdx.x; r < nb; r += kBV) {
      const double v = __ldcg(w + a0 + r) * inv;
      w[a0 + r] = v;
      if (a.bj64)
        wsd[r] = v;
      else
        ws[r] = (float)v;
    }
    __syncthreads();
    if (a.bj64)
      bj_body_apply64(a.blocks + a.off[i], nb, wsd, a.z + a0);
    else
      bj_body_apply(a.blocks + a.off[i], a.off[i], nb, ws, a.z + a0, red4);
    __syncthreads();
  }
}

// ------------------------------------------- Arnoldi step of the FP32 solves
// The inner solves of the refinement apply the operator in FP32 and stop at a
// relative residual of about 1e-6, so their Krylov basis needs FP32
// orthogonality only.  This step runs CGS2 in FP32 arithmetic against an
// FP32 copy VF of the basis (v_i as the floats the preconditioner and the
// operator already see): rounding w = A z_j to FP32 and the FP32 projections
// perturb the Arnoldi relation A P V = V H by O(eps32 ||w||), the size of the
// FP32 operator's own error, and the second pass restores orthogonality to
// O(eps32) (classical Gram-Schmidt twice).  The FP64 path above spends 4(j+1)
// FP64 multiply-adds an element on GB300's narrow FP64 pipe (two lanes a
// clock per SM); this one 4(j+1) FP32 ones, and reads half the bytes.
// Threads own chunks of four consecutive elements (16-byte loads; VF rows
// are 16-byte aligned and padded to ld, the padding of the chunk at the end
// holds zeros).  The per-CTA partials and the grid sums are FP32 too (sums of
// FP32 dot products, in a fixed order: deterministic); the Hessenberg column
// and the rotations stay in FP64.  V_{j+1} (FP64, read by the solution
// update) receives the FP32 basis vector exactly.

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}

constexpr int kDot32 = 4;  // basis vectors a pass of the FP32 inner products

// Partial dot products of this CTA's chunks of x with VF_0..VF_{jc-1} into
// out[0..jc): kDot32 basis vectors a pass, FP32 sums per thread, a fixed
// shuffle tree per warp, the warps added in order.
__device__ __forceinline__ void arn_block_dots32(const float* __restrict__ VF, long long ld,
                                                 const float* __restrict__ x, long long n4, int jc,
                                                 float* __restrict__ out, float (*sh)[kMaxBasis]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long stride = (long long)gridDim.x * kBV;
  const long long ld4 = ld >> 2;
  const float4* __restrict__ V4 = reinterpret_cast<const float4*>(VF);
  const float4* __restrict__ x4 = reinterpret_cast<const float4*>(x);
  for (int i = 0; i < jc; i += kDot32) {
    const int cnt = min(kDot32, jc - i);
    float acc[kDot32];
#pragma unroll
    for (int u = 0; u < kDot32; ++u) acc[u] = 0.f;
    for (long long c = blockIdx.x * (long long)kBV + threadIdx.x; c < n4; c += stride) {
      const float4 xc = x4[c];
#pragma unroll
      for (int u = 0; u < kDot32; ++u)
        if (u < cnt) acc[u] = dot4(V4[(long long)(i + u) * ld4 + c], xc, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < kDot32; ++u) {
      if (u < cnt) {
        const float t = warp_sumf(acc[u]);
        if (lane == 0) sh[wid][i + u] = t;
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < jc; q += kBV) {
    float t = 0.f;
#pragma unroll
    for (int u = 0; u < kBV / 32; ++u) t += sh[u][q];
    out[q] = t;
  }
}

// hs[i] = sum over CTAs b of part[b * kMaxBasis + i] (FP32 partials written
// by other CTAs before a grid barrier; read through L2), i < jc: warp u takes
// i = u, u + 8, ...; its lanes take b = lane, lane + 32, ... with four
// independent sums (loads in flight), then a fixed shuffle tree.
__device__ __forceinline__ void arn_grid_sum32(const float* part, int jc, double* hs) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int G = (int)gridDim.x;
  for (int i = wid; i < jc; i += kBV / 32) {
    float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
    int b = lane;
    for (; b + 96 < G; b += 128) {
      t0 += __ldcg(part + (long long)b * kMaxBasis + i);
      t1 += __ldcg(part + (long long)(b + 32) * kMaxBasis + i);
      t2 += __ldcg(part + (long long)(b + 64) * kMaxBasis + i);
      t3 += __ldcg(part + (long long)(b + 96) * kMaxBasis + i);
    }
    for (; b < G; b += 32) t0 += __ldcg(part + (long long)b * kMaxBasis + i);
    const float t = warp_sumf((t0 + t1) + (t2 + t3));
    if (lane == 0) hs[i] = (double)t;
  }
  __syncthreads();
}

// x -= VF h over this CTA's chunks (two FP32 chains, fixed order); returns
// this thread's FP32 sum of the new x^2 when NORM.
template <bool NORM>
__device__ __forceinline__ float arn_project32(const float* __restrict__ VF, long long ld, float* __restrict__ x,
                                               long long n4, int jc, const float* h) {
  const long long stride = (long long)gridDim.x * kBV;
  const long long ld4 = ld >> 2;
  const float4* __restrict__ V4 = reinterpret_cast<const float4*>(VF);
  float4* __restrict__ x4 = reinterpret_cast<float4*>(x);
  float nrm = 0.f;
  for (long long c = blockIdx.x * (long long)kBV + threadIdx.x; c < n4; c += stride) {
    float4 t0 = x4[c], t1 = make_float4(0.f, 0.f, 0.f, 0.f);
    int i = 0;
    for (; i + 2 <= jc; i += 2) {
      const float4 a = V4[(long long)i * ld4 + c], b = V4[(long long)(i + 1) * ld4 + c];
      const float ha = -h[i], hb = -h[i + 1];
      t0 = make_float4(fmaf(ha, a.x, t0.x), fmaf(ha, a.y, t0.y), fmaf(ha, a.z, t0.z), fmaf(ha, a.w, t0.w));
      t1 = make_float4(fmaf(hb, b.x, t1.x), fmaf(hb, b.y, t1.y), fmaf(hb, b.z, t1.z), fmaf(hb, b.w, t1.w));
    }
    if (i < jc) {
      const float4 a = V4[(long long)i * ld4 + c];
      const float ha = -h[i];
      t0 = make_float4(fmaf(ha, a.x, t0.x), fmaf(ha, a.y, t0.y), fmaf(ha, a.z, t0.z), fmaf(ha, a.w, t0.w));
    }
    const float4 t = make_float4(t0.x + t1.x, t0.y + t1.y, t0.z + t1.z, t0.w + t1.w);
    x4[c] = t;
    if (NORM) nrm = dot4(t, t, nrm);
  }
  return nrm;
}

__global__ void __launch_bounds__(kBV, 4) k_arnoldi32(ArnoldiArgs a) {
  KState* st = a.st;
  if (st->stop) return;  // read by every CTA before the first barrier: uniform
  __shared__ float shf[kBV / 32][kMaxBasis];
  __shared__ double hs1[kMaxBasis], hs2[kMaxBasis];
  __shared__ float hf[kMaxBasis];
  __shared__ float redf[kBV / 32];
  __shared__ float ws[kBjMaxBlock];
  __shared__ float4 red4[2 * kBV];
  const int j = st->j, jc = j + 1;
  const long long n = a.n, ld = a.ld, n4 = (n + 3) >> 2;
  float* __restrict__ VF = a.vf;
  double* __restrict__ w = a.V + (long long)(j + 1) * ld;  // A z_j (FP64, from the operator)
  float* __restrict__ wf = VF + (long long)(j + 1) * ld;    // w in FP32, then v_{j+1}
  const long long stride = (long long)gridDim.x * kBV;
  const long long G = gridDim.x;
  // FP32 partials in the partial arrays: [G][kMaxBasis] floats each
  float* part1 = reinterpret_cast<float*>(a.part);
  float* part2 = part1 + G * kMaxBasis;
  float* part3 = part2 + G * kMaxBasis;
  // VF_j = V_j in FP32 (exact for j > 0: V_j came from VF_j), w in FP32; the
  // padding after element n of the last chunk set to zero
  {
    const double* __restrict__ vj = a.V + (long long)j * ld;
    float4* __restrict__ vfj4 = reinterpret_cast<float4*>(VF + (long long)j * ld);
    float4* __restrict__ wf4 = reinterpret_cast<float4*>(wf);
    for (long long c = blockIdx.x * (long long)kBV + threadIdx.x; c < n4; c += stride) {
      const long long k = 4 * c;
      float4 vv, ww;
      if (k + 4 <= n) {
        const double2 v0 = *reinterpret_cast<const double2*>(vj + k), v1 = *reinterpret_cast<const double2*>(vj + k + 2);
        const double2 w0 = *reinterpret_cast<const double2*>(w + k), w1 = *reinterpret_cast<const double2*>(w + k + 2);
        vv = make_float4((float)v0.x, (float)v0.y, (float)v1.x, (float)v1.y);
        ww = make_float4((float)w0.x, (float)w0.y, (float)w1.x, (float)w1.y);
      } else {
        float vt[4], wt[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          vt[e] = k + e < n ? (float)vj[k + e] : 0.f;
          wt[e] = k + e < n ? (float)w[k + e] : 0.f;
        }
        vv = make_float4(vt[0], vt[1], vt[2], vt[3]);
        ww = make_float4(wt[0], wt[1], wt[2], wt[3]);
      }
      vfj4[c] = vv;
      wf4[c] = ww;
    }
  }
  // h1 = VF^T w
  arn_block_dots32(VF, ld, wf, n4, jc, part1 + blockIdx.x * kMaxBasis, shf);
  if ((int)blockIdx.x == a.fault_skip) return;  // test hook: this CTA never arrives
  if (grid_barrier(st, a.spins)) return;
  arn_grid_sum32(part1, jc, hs1);
  for (int i = threadIdx.x; i < jc; i += kBV) hf[i] = (float)hs1[i];
  __syncthreads();
  // w -= VF h1; h2 = VF^T w
  arn_project32<false>(VF, ld, wf, n4, jc, hf);
  __syncthreads();  // hf and shf are reused below
  arn_block_dots32(VF, ld, wf, n4, jc, part2 + blockIdx.x * kMaxBasis, shf);
  if (grid_barrier(st, a.spins)) return;
  arn_grid_sum32(part2, jc, hs2);
  for (int i = threadIdx.x; i < jc; i += kBV) hf[i] = (float)hs2[i];
  __syncthreads();
  // w -= VF h2; ||w||^2
  float nrm = arn_project32<true>(VF, ld, wf, n4, jc, hf);
  nrm = warp_sumf(nrm);
  if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
#pragma unroll
    for (int u = 0; u < kBV / 32; ++u) t += redf[u];
    part3[blockIdx.x * kMaxBasis] = t;
  }
  if (grid_barrier(st, a.spins)) return;
  __shared__ double hn2[1];
  arn_grid_sum32(part3, 1, hn2);
  const double hn = sqrt(hn2[0]);
  if (blockIdx.x == 0) arn_hessenberg(a, st, j, hs1, hs2, hn);
  const float inv = hn > 0.0 ? (float)(1.0 / hn) : 0.f;
  if (!a.blocks) {
    // v_{j+1} = w / ||w|| over this CTA's own elements
    for (long long c = blockIdx.x * (long long)kBV + threadIdx.x; c < n4; c += stride) {
      for (int e = 0; e < 4; ++e) {
        const long long k = 4 * c + e;
        if (k < n) {
          const float v = wf[k] * inv;
          wf[k] = v;
          w[k] = (double)v;
        }
      }
    }
    return;
  }
  // per body: v = w inv (w read through L2: other CTAs wrote it), z = P v.
  // CTA 0 computes the Hessenberg column and rotations above, so the bodies
  // go to CTAs 1..G-1 (with one CTA, to CTA 0).
  const int c = a.kind + 1;
  const int first = G > 1 ? (int)blockIdx.x - 1 : 0, nworkers = G > 1 ? (int)G - 1 : 1;
  if (first < 0) return;
  for (int i = first; i < a.g.N; i += nworkers) {
    const long long a0 = (long long)a.g.body_start[i] * c;
    const int nb = (a.g.body_start[i + 1] - a.g.body_start[i]) * c;
    const bool apply = nb <= kBjMaxBlock;
    for (int r = threadIdx.x; r < nb; r += kBV) {
      const float v = __ldcg(wf + a0 + r) * inv;
      wf[a0 + r] = v;
      w[a0 + r] = (double)v;
      if (apply)
        ws[r] = v;
      else
        a.z[a0 + r] = (double)v;
    }
    if (!apply) continue;
    __syncthreads();
    bj_body_apply(a.blocks + a.off[i], a.off[i], nb, ws, a.z + a0, red4);
    __syncthreads();
  }
}

// ------------------------------------------------------ batched Arnoldi
// The fused Arnoldi step of many independent problems (one block-diagonal
// system, each problem its own Krylov space).  The vector is cut into element
// ranges that never cross a problem; CTA b takes ranges b, b + G, ...  The
// inner products of a problem add the per-range partials of that problem's
// ranges in range order (deterministic).  Problem p takes part in step j while
// stop_j > j; its Givens rotations run on CTA p mod G.  A problem that stopped
// earlier is skipped and its next basis vector set to zero, so that the
// operator applied to it gives zero.

// Partial dot products of w[e0, e1) with V_0..V_{jc-1} into out[0..jc):
// warp u takes basis vectors u, u + 8, ..., its lanes stride the range with
// two independent sums (fixed order: deterministic).
__device__ __forceinline__ void seg_block_dots(const double* __restrict__ V, long long ld, const double* __restrict__ w,
                                               long long e0, long long e1, int jc, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < jc; i += kBV / 32) {
    const double* __restrict__ Vi = V + (long long)i * ld;
    double a0 = 0.0, a1 = 0.0;
    long long k = e0 + lane;
    for (; k + 32 < e1; k += 64) {
      a0 = fma(Vi[k], w[k], a0);
      a1 = fma(Vi[k + 32], w[k + 32], a1);
    }
    if (k < e1) a0 = fma(Vi[k], w[k], a0);
    const double t = warp_sum(a0 + a1);
    if (lane == 0) out[i] = t;
  }
  __syncthreads();
}

// hs[i] = sum over the ranges [it0, it1) of part[it][i] (written by other CTAs
// before a grid barrier; read through L2), i < jc.
__device__ __forceinline__ void seg_sum(const double* part, int it0, int it1, int jc, double* hs) {
  __syncthreads();  // hs may still be read from the previous range
  for (int i = threadIdx.x; i < jc; i += kBV) {
    double t = 0.0;
#pragma unroll 4
    for (int it = it0; it < it1; ++it) t += __ldcg(part + (long long)it * kMaxBasis + i);
    hs[i] = t;
  }
  __syncthreads();
}

// ||w_p|| after orthogonalisation: the sum of the range partials, broadcast.
__device__ __forceinline__ double seg_hn(const double* part3, int it0, int it1, double* cell) {
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int it = it0; it < it1; ++it) t += __ldcg(part3 + (long long)it * kMaxBasis);
    *cell = sqrt(t);
  }
  __syncthreads();
  return *cell;
}

__global__ void __launch_bounds__(kBV) k_arnoldi_seg(ArnoldiArgs a, SegArgs sg) {
  KState* st = a.st;
  if (st->stop) return;  // read by every CTA before the first barrier: uniform
  __shared__ double hs[kMaxBasis], hcol[kMaxBasis + 1];
  __shared__ double red[kBV / 32];
  __shared__ double cell;
  __shared__ float ws[kBjMaxBlock];
  __shared__ double wsd[kBjMaxBlock];
  __shared__ float4 red4[2 * kBV];
  const int j = st->j, jc = j + 1;
  const long long ld = a.ld;
  double* __restrict__ w = a.V + (long long)(j + 1) * ld;
  const int G = gridDim.x;
  double* part1 = a.part;
  double* part2 = part1 + (long long)sg.nitem * kMaxBasis;
  double* part3 = part2 + (long long)sg.nitem * kMaxBasis;
  // h1 = V^T w per range
  for (int it = blockIdx.x; it < sg.nitem; it += G) {
    const int p = sg.iprob[it];
    if (sg.ps[p].stop_j <= j) continue;
    seg_block_dots(a.V, ld, w, sg.ibeg[it], sg.ibeg[it + 1], jc, part1 + (long long)it * kMaxBasis);
  }
  if ((int)blockIdx.x == a.fault_skip) return;  // test hook: this CTA never arrives
  if (grid_barrier(st, a.spins)) return;
  // w -= V h1; h2 = V^T w
  for (int it = blockIdx.x; it < sg.nitem; it += G) {
    const int p = sg.iprob[it];
    if (sg.ps[p].stop_j <= j) continue;
    seg_sum(part1, sg.pitem[p], sg.pitem[p + 1], jc, hs);
    const long long e0 = sg.ibeg[it], e1 = sg.ibeg[it + 1];
    for (long long k = e0 + threadIdx.x; k < e1; k += kBV) w[k] = w[k] - combine(a.V, ld, k, hs, jc);
    __syncthreads();
    seg_block_dots(a.V, ld, w, e0, e1, jc, part2 + (long long)it * kMaxBasis);
  }
  if (grid_barrier(st, a.spins)) return;
  // w -= V h2; ||w||^2 per range
  for (int it = blockIdx.x; it < sg.nitem; it += G) {
    const int p = sg.iprob[it];
    if (sg.ps[p].stop_j <= j) continue;
    seg_sum(part2, sg.pitem[p], sg.pitem[p + 1], jc, hs);
    const long long e0 = sg.ibeg[it], e1 = sg.ibeg[it + 1];
    double nrm = 0.0;
    for (long long k = e0 + threadIdx.x; k < e1; k += kBV) {
      const double t = w[k] - combine(a.V, ld, k, hs, jc);
      w[k] = t;
      nrm = fma(t, t, nrm);
    }
    nrm = block_sum<kBV>(nrm, red);
    if (threadIdx.x == 0) part3[(long long)it * kMaxBasis] = nrm;
  }
  if (grid_barrier(st, a.spins)) return;
  // Hessenberg column, rotations and stopping test of each problem
  const int m = st->m;
  for (int p = blockIdx.x; p < sg.P; p += G) {
    PState* q = sg.ps + p;
    if (q->stop_j <= j) continue;
    const int it0 = sg.pitem[p], it1 = sg.pitem[p + 1];
    seg_sum(part1, it0, it1, jc, hs);
    for (int i = threadIdx.x; i < jc; i += kBV) hcol[i] = hs[i];
    seg_sum(part2, it0, it1, jc, hs);
    for (int i = threadIdx.x; i < jc; i += kBV) hcol[i] += hs[i];
    const double hn = seg_hn(part3, it0, it1, &cell);
    double* Hc = a.H + (long long)p * (m + 1) * m + (long long)j * (m + 1);
    double* cs = a.cs + (long long)p * m;
    double* sn = a.sn + (long long)p * m;
    double* gv = a.gv + (long long)p * (m + 1);
    if (threadIdx.x == 0) {
      hcol[j + 1] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t;
      }
      const double x = hcol[j], y = hcol[j + 1];
      const double r = hypot(x, y);
      const double c = r > 0.0 ? x / r : 1.0, sgn = r > 0.0 ? y / r : 0.0;
      cs[j] = c;
      sn[j] = sgn;
      hcol[j] = r;
      hcol[j + 1] = 0.0;
      const double g = gv[j];
      gv[j + 1] = -sgn * g;
      gv[j] = c * g;
      q->res = fabs(sgn * g);
      if (q->res <= q->tol_abs || !(hn > 1e-300 * q->beta)) {
        q->stop_j = j + 1;
        if (atomicSub(&st->nactive, 1) == 1) st->stop = 1;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= j + 1; i += kBV) Hc[i] = hcol[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->j = j + 1;
    st->iters += 1;
    if (j + 1 >= m || st->iters >= st->maxit) st->stop = 1;
  }
  // v_{j+1} = w / ||w|| per problem (zero for a problem that stopped before
  // this step); with the preconditioner also z = P v, per body
  if (!a.blocks) {
    for (int it = blockIdx.x; it < sg.nitem; it += G) {
      const int p = sg.iprob[it];
      const bool active = sg.ps[p].stop_j > j;  // stop_j is j + 1 or above if set in this step
      const double hn = active ? seg_hn(part3, sg.pitem[p], sg.pitem[p + 1], &cell) : 0.0;
      const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
      for (long long k = sg.ibeg[it] + threadIdx.x; k < sg.ibeg[it + 1]; k += kBV) w[k] = active ? w[k] * inv : 0.0;
    }
    return;
  }
  const int c = a.kind + 1;
  for (int i = blockIdx.x; i < a.g.N; i += G) {
    const int p = sg.bprob[i];
    const long long a0 = (long long)a.g.body_start[i] * c;
    const int nb = (a.g.body_start[i + 1] - a.g.body_start[i]) * c;
    const bool active = sg.ps[p].stop_j > j;
    const double hn = active ? seg_hn(part3, sg.pitem[p], sg.pitem[p + 1], &cell) : 0.0;
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    if (!active || nb > kBjMaxBlock) {
      for (int r = threadIdx.x; r < nb; r += kBV) {
        const double v = active ? __ldcg(w + a0 + r) * inv : 0.0;
        w[a0 + r] = v;
        a.z[a0 + r] = v;
      }
      continue;
    }
    __syncthreads();  // ws may still be read for the previous body
    for (int r = threadIdx.x; r < nb; r += kBV) {
      const double v = __ldcg(w + a0 + r) * inv;
      w[a0 + r] = v;
      if (a.bj64)
        wsd[r] = v;
      else
        ws[r] = (float)v;
    }
    __syncthreads();
    if (a.bj64)
      bj_body_apply64(a.blocks + a.off[i], nb, wsd, a.z + a0);
    else
      bj_body_apply(a.blocks + a.off[i], a.off[i], nb, ws, a.z + a0, red4);
  }
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
  if (!is_last || threadIdx.x >= 32) return;
  __threadfence();
  const double s = warp_gather(part, 1);
  if (threadIdx.x != 0) return;
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

// Batched GMRES, one CTA per problem: r = f - y over the problem's entries,
// its norm, and the opening of a cycle (g_p = (||r_p||, 0, ..); the problem
// takes part unless already below its tolerance).  On the first call of a
// solve (st->pad[0]) the tolerance is set relative to ||r_p|| = ||b_p||.  The
// last CTA counts the active problems and stops the cycle if there are none.
__global__ void __launch_bounds__(kBV) k_residual_seg(const double* __restrict__ f, const double* __restrict__ y,
                                                      double* __restrict__ r, KState* st, SegArgs sg,
                                                      double* gv, int m) {
  __shared__ double sh[kBV / 32];
  __shared__ int is_last;
  const int p = blockIdx.x;
  const long long k0 = sg.pnode[p], k1 = sg.pnode[p + 1];
  double nrm = 0.0;
  for (long long k = k0 + threadIdx.x; k < k1; k += kBV) {
    const double v = y ? f[k] - y[k] : f[k];
    r[k] = v;
    nrm += v * v;
  }
  nrm = block_sum<kBV>(nrm, sh);
  if (threadIdx.x == 0) {
    PState* q = sg.ps + p;
    const double rn = sqrt(nrm);
    if (st->pad[0]) {
      q->tol_abs = st->scratch[0] * rn;
      q->bnorm = rn;
    }
    q->rnorm = rn;
    q->beta = rn;
    q->res = rn;
    gv[(long long)p * (m + 1)] = rn;
    q->stop_j = (rn <= q->tol_abs || !(rn > 0.0)) ? 0 : 0x7fffffff;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!is_last || threadIdx.x >= 32) return;
  __threadfence();
  int cnt = 0;
  double s2 = 0.0;
  for (int q = threadIdx.x; q < sg.P; q += 32) {
    const double rn = __ldcg(&sg.ps[q].rnorm);
    s2 += rn * rn;
    cnt += __ldcg(&sg.ps[q].stop_j) > 0 ? 1 : 0;
  }
  s2 = warp_sum(s2);
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (threadIdx.x != 0) return;
  st->counter = 0;
  st->pad[0] = 0;
  st->rnorm = sqrt(s2);
  st->nactive = cnt;
  st->j = 0;
  st->stop = (cnt == 0 || st->iters >= st->maxit) ? 1 : 0;
}

// V_0 = r / beta_p per problem (blockIdx.y = p; zero if the problem does not
// take part in the cycle).
__global__ void k_start_v0_seg(const double* __restrict__ r, double* __restrict__ V0, const KState* st,
                               SegArgs sg) {
  if (st->stop) return;
  const int p = blockIdx.y;
  const PState& q = sg.ps[p];
  const double inv = q.stop_j > 0 ? 1.0 / q.beta : 0.0;
  for (long long k = sg.pnode[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < sg.pnode[p + 1];
       k += (long long)gridDim.x * blockDim.x)
    V0[k] = r[k] * inv;
}

// y_p = R_p^{-1} g_p over the steps problem p took part in (one thread each).
__global__ void k_triangular_seg(const KState* st, SegArgs sg, const double* __restrict__ H,
                                 const double* __restrict__ gv, double* y, int m) {
  const int p = blockIdx.x;
  if (threadIdx.x != 0) return;
  const int jp = min(sg.ps[p].stop_j, st->j);
  const double* Hp = H + (long long)p * (m + 1) * m;
  const double* gp = gv + (long long)p * (m + 1);
  double* yp = y + (long long)p * (m + 1);
  for (int i = jp - 1; i >= 0; --i) {
    double s = gp[i];
    for (int k = i + 1; k < jp; ++k) s -= Hp[(long long)k * (m + 1) + i] * yp[k];
    yp[i] = s / Hp[(long long)i * (m + 1) + i];
  }
}

// x += V y_p over problem p's entries (blockIdx.y = p).
__global__ void k_update_x_seg(const double* __restrict__ V, long long ld, const KState* st, SegArgs sg,
                               const double* __restrict__ y, double* __restrict__ x, int m) {
  __shared__ double ys[kMaxBasis];
  const int p = blockIdx.y;
  const int jp = min(sg.ps[p].stop_j, st->j);
  if (jp <= 0) return;
  for (int i = threadIdx.x; i < jp; i += blockDim.x) ys[i] = y[(long long)p * (m + 1) + i];
  __syncthreads();
  for (long long k = sg.pnode[p] + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < sg.pnode[p + 1];
       k += (long long)gridDim.x * blockDim.x)
    x[k] += combine(V, ld, k, ys, jp);
}

inline int elt_grid(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

}  // namespace

int vec_grid(long long n) {
  long long b = (n + kBV - 1) / kBV;
  if (b > kMaxVecGrid) b = kMaxVecGrid;
  if (b < 1) b = 1;
  return (int)b;
}

// The narrow instance for grids of at most two CTAs per SM.
bool arnoldi_narrow(long long n) { return vec_grid(n) <= 2 * device_sms(); }

int arnoldi_grid(long long n, bool fp32, int nbodies) {
  static std::atomic<int> coresident[64][3];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  const int narrow = arnoldi_narrow(n) ? 1 : 0;
  const int v = fp32 ? 2 : (narrow ? 1 : 0);
  if (coresident[dev][v].load() == 0) {
    int per_sm = 0, sms = 0;
    const void* fn = v == 1 ? (const void*)k_arnoldi<true> : (v == 2 ? (const void*)k_arnoldi32 : (const void*)k_arnoldi<false>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBV, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm * sms < 1) {
      cudaGetLastError();
      return 1;  // not cached: a launch of one CTA is always co-resident
    }
    coresident[dev][v].store(per_sm * sms);
  }
  // the FP32 step gives CTA 0 the rotations and CTAs 1.. the bodies: at least
  // one CTA a body where the grid allows
  const int want = fp32 ? std::max(vec_grid(n), std::min(nbodies + 1, kMaxVecGrid)) : vec_grid(n);
  return std::min(want, coresident[dev][v].load());
}

namespace {
// Test hook of the bounded barrier waits (bie_test_arm_barrier_timeout): taken
// by the next Arnoldi launch only.
std::atomic<long long> g_fault_spins{0};
std::atomic<int> g_fault_skip{-1};

void take_fault(ArnoldiArgs& args) {
  const long long sp = g_fault_spins.exchange(0);
  if (sp > 0) {
    args.fault_skip = g_fault_skip.load();
    args.spins = sp;
  } else {
    args.fault_skip = -1;
    args.spins = kBarrierSpins;
  }
}
}  // namespace

void arm_barrier_fault(int skip_cta, long long spins) {
  g_fault_skip.store(skip_cta);
  g_fault_spins.store(spins > 0 ? spins : 0);
}

bool barrier_fault_armed() { return g_fault_spins.load() > 0; }

cudaError_t arnoldi(const ArnoldiArgs& a, int grid, cudaStream_t s) {
  ArnoldiArgs args = a;
  take_fault(args);
  void* params[] = {&args};
  const void* fn = a.vf ? (const void*)k_arnoldi32
                        : (arnoldi_narrow(a.n) ? (const void*)k_arnoldi<true> : (const void*)k_arnoldi<false>);
  const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBV), params, 0, s);
  note_launches(1);
  return e;
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

int arnoldi_seg_grid(long long n) {
  static std::atomic<int> coresident[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (coresident[dev].load() == 0) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_arnoldi_seg, kBV, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm * sms < 1) {
      cudaGetLastError();
      return 1;
    }
    coresident[dev].store(per_sm * sms);
  }
  return std::min(vec_grid(n), coresident[dev].load());
}

cudaError_t arnoldi_seg(const ArnoldiArgs& a, const SegArgs& sg, int grid, cudaStream_t s) {
  ArnoldiArgs args = a;
  take_fault(args);
  SegArgs sargs = sg;
  void* params[] = {&args, &sargs};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_arnoldi_seg, dim3(grid), dim3(kBV), params, 0, s);
  note_launches(1);
  return e;
}

cudaError_t residual_start_seg(const double* f, const double* y, double* r, double* V0, KState* st,
                               const SegArgs& sg, double* gv, int m, cudaStream_t s) {
  k_residual_seg<<<sg.P, kBV, 0, s>>>(f, y, r, st, sg, gv, m);
  note_launches(1);
  k_start_v0_seg<<<dim3(8, sg.P), 256, 0, s>>>(r, V0, st, sg);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t gmres_update_seg(const double* V, long long ld, KState* st, const SegArgs& sg, const double* H,
                             const double* gv, double* y, double* x, int m, long long max_len, cudaStream_t s) {
  k_triangular_seg<<<sg.P, 32, 0, s>>>(st, sg, H, gv, y, m);
  note_launches(1);
  const long long bx = std::min<long long>(64, std::max<long long>(1, (max_len + 255) / 256));
  k_update_x_seg<<<dim3((unsigned)bx, sg.P), 256, 0, s>>>(V, ld, st, sg, y, x, m);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bie
