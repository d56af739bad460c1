// Nystrom pair sums of the paper's second-kind operators and their epilogue.
//
// Laplace (Section 3.4, operator K with the TARGET normal):
//   (K mu)_a = -(1/2pi) sum_{b != a} w_b mu_b (r . n_a) / |r|^2,   r = x_a - x_b
// Stokes (Section 4.3, operator K built from the stresslet T_ijk = -(1/pi) r_i r_j r_k/|r|^4):
//   (K mu)_a = -(1/pi) sum_{b != a} w_b r (r . mu_b)(r . n_a) / |r|^4
//
// Layout of the work: a block owns B*T targets (T per thread, strided by B so
// loads coalesce) and one contiguous split of the sources; sources stream
// through shared memory in tiles.  The splits write partial sums
// partial[s][a] that the epilogue adds in a fixed order (deterministic), in
// FP64, together with the diagonal limit, 1/2 I and the completion L.
//
// FP32 variant: positions are held as hi/lo float pairs so that, for a source
// tile close to the target block, dx = (xa_hi - xb_hi) + (xa_lo - xb_lo) is
// exact to FP32 rounding of dx itself even for neighbouring nodes far from the
// origin (the near-pair cancellation in r . n_a would otherwise lose digits).
// Tiles far from the block (gap at least both boxes' half-diagonals) use plain
// FP32 coordinates relative to the block centre: 4 fewer instructions a pair.
// The reciprocal is the hardware rcp.approx.f32; tile sums enter
// TwoSum-compensated FP32 accumulators.  The per-pair arithmetic (FP32 near
// pairs and float-float pairs) is shared with the FMM near field.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "bie_internal.cuh"
#include "pair_math.cuh"
#include "reduce.cuh"

namespace bie {

namespace {

// Source range of a target block [tbase, tend): all nodes, or in a batch the
// nodes of the problems its targets belong to (straddle: more than one); the
// block's split blockIdx.y of it, `chunk` sources long.  In a batch the range
// is cut into chunks of the planned length, so a block of a small problem has
// fewer busy splits than one of a large problem (the others are empty and
// write zero partials); a range longer than all splits together (a block
// straddling problems) is cut into gridDim.y equal parts.
struct SrcRange {
  int j0, j1;
  bool straddle;
};

template <bool BATCH>
__device__ __forceinline__ SrcRange src_range(const Geo& g, int tbase, int tend, const PairPlan& p) {
  SrcRange r;
  if (!BATCH) {
    const int s = blockIdx.y;
    r.j0 = s < p.S1 ? s * p.chunk : p.S1 * p.chunk + (s - p.S1) * p.chunk2;
    r.j1 = min(g.M, r.j0 + (s < p.S1 ? p.chunk : p.chunk2));
    r.straddle = false;
    return r;
  }
  const int chunk = p.chunk;
  const int2 p0 = g.prange[g.body_of[tbase]], p1 = g.prange[g.body_of[tend - 1]];
  const int len = p1.y - p0.x;
  const int ch = max(chunk, (len + (int)gridDim.y - 1) / (int)gridDim.y);
  r.j0 = min(p1.y, p0.x + (int)blockIdx.y * ch);
  r.j1 = min(p1.y, r.j0 + ch);
  r.straddle = p0.x != p1.x;
  return r;
}

// Batched GMRES: have all problems of the target block [tbase, tend) stopped?
// (block-uniform)  Such a block writes zero partials: its problems' next
// Krylov vectors are not used.
__device__ __forceinline__ bool block_stopped(const Geo& g, int tbase, int tend) {
  if (!g.ps) return false;
  const int j = *g.jstep;
  const int p0 = g.bprob[g.body_of[tbase]], p1 = g.bprob[g.body_of[tend - 1]];
  for (int p = p0; p <= p1; ++p)
    if (g.ps[p].stop_j > j) return false;
  return true;
}

template <int KIND>
__device__ __forceinline__ void zero_partials(int tbase, int tend, int M, double* __restrict__ partial) {
  for (int a = tbase + threadIdx.x; a < tend; a += blockDim.x) {
    if (KIND == 0) {
      partial[(long long)blockIdx.y * M + a] = 0.0;
    } else {
      partial[((long long)blockIdx.y * M + a) * 2] = 0.0;
      partial[((long long)blockIdx.y * M + a) * 2 + 1] = 0.0;
    }
  }
}

// Does source node b belong to target a's problem (batched solves)?
__device__ __forceinline__ bool same_problem(const Geo& g, int a, int b) {
  if (a >= g.M) return true;
  const int2 r = g.prange[g.body_of[a]];
  return b >= r.x && b < r.y;
}

// End of the tile starting at source jt: at most `want`, cut at the end of
// jt's problem (a tile must not mix problems).
template <bool BATCH>
__device__ __forceinline__ int tile_len(const Geo& g, int jt, int want) {
  if (!BATCH) return want;
  return min(want, g.prange[g.body_of[jt]].y - jt);
}

// ------------------------------------------------------------------ FP64 ----
constexpr int kB64 = 128, kT64 = 2, kTile64 = 128;

template <int KIND, bool BATCH>
__global__ void __launch_bounds__(kB64) k_pair64(Geo g, VecRef vr, const double* __restrict__ sscale,
                                                 PairPlan pp, double* __restrict__ partial,
                                                 const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double sx[kTile64], sy[kTile64], sq1[kTile64], sq2[kTile64];
  const double* __restrict__ v = vr.ptr();
  const int M = g.M;
  const int tbase = blockIdx.x * kB64 * kT64;
  if (BATCH && block_stopped(g, tbase, min(M, tbase + kB64 * kT64))) {
    zero_partials<KIND>(tbase, min(M, tbase + kB64 * kT64), M, partial);
    return;
  }
  const SrcRange sr = src_range<BATCH>(g, tbase, min(M, tbase + kB64 * kT64), pp);
  const int j0 = sr.j0, j1 = sr.j1;
  double tx[kT64], ty[kT64], tnx[kT64], tny[kT64], ax[kT64], ay[kT64];
  int ta[kT64];
#pragma unroll
  for (int k = 0; k < kT64; ++k) {
    const int a = tbase + threadIdx.x + k * kB64;
    ta[k] = a;
    const bool in = a < M;
    tx[k] = in ? g.x[a] : 0.0;
    ty[k] = in ? g.y[a] : 0.0;
    tnx[k] = in ? g.nx[a] : 0.0;
    tny[k] = in ? g.ny[a] : 0.0;
    ax[k] = 0.0;
    ay[k] = 0.0;
  }
  for (int jt = j0; jt < j1; jt += kTile64) {
    __syncthreads();
    for (int l = threadIdx.x; l < kTile64; l += kB64) {
      const int b = jt + l;
      if (b < j1) {
        sx[l] = g.x[b];
        sy[l] = g.y[b];
        if (KIND == 0) {
          sq1[l] = sscale[b] * v[b];
        } else {
          sq1[l] = sscale[b] * v[2 * b];
          sq2[l] = sscale[b] * v[2 * b + 1];
        }
      }
    }
    __syncthreads();
    const int nt = min(kTile64, j1 - jt);
    for (int l = 0; l < nt; ++l) {
      const double px = sx[l], py = sy[l], q1 = sq1[l];
      const double q2 = KIND == 0 ? 0.0 : sq2[l];
      const int b = jt + l;
#pragma unroll
      for (int k = 0; k < kT64; ++k) {
        const double dx = tx[k] - px, dy = ty[k] - py;
        const double r2 = dx * dx + dy * dy;
        const bool skip = ta[k] == b || (BATCH && sr.straddle && !same_problem(g, ta[k], b));
        if (KIND == 0) {
          const double s = skip ? 0.0 : q1 / r2;
          ax[k] += dx * s;
          ay[k] += dy * s;
        } else {
          const double rq = dx * q1 + dy * q2;
          const double rn = dx * tnx[k] + dy * tny[k];
          const double c = skip ? 0.0 : (rq * rn) / (r2 * r2);
          ax[k] += c * dx;
          ay[k] += c * dy;
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kT64; ++k) {
    const int a = ta[k];
    if (a < M) {
      if (KIND == 0)
        partial[(long long)blockIdx.y * M + a] = tnx[k] * ax[k] + tny[k] * ay[k];
      else {
        partial[((long long)blockIdx.y * M + a) * 2] = ax[k];
        partial[((long long)blockIdx.y * M + a) * 2 + 1] = ay[k];
      }
    }
  }
}

// ------------------------------------------------------------------ FP32 ----
constexpr int kB32 = 64, kT32 = 4, kTile32 = 256;

// Near tiles (sources whose bounding box is close to the target block's):
// exact differences from the hi/lo coordinates, reloaded here so that they
// are not live across the far tiles.
template <int KIND, bool DIAG>
__device__ __forceinline__ void tile_near(const float4* __restrict__ pf, const float4* __restrict__ sp,
                                          const float2* __restrict__ sq, int nt, int jt, int a0, int M,
                                          const float* tnx, const float* tny, float* ax, float* ay) {
  float txh[kT32], tyh[kT32], txl[kT32], tyl[kT32];
#pragma unroll
  for (int k = 0; k < kT32; ++k) {
    const int a = a0 + k * kB32;
    const float4 p = a < M ? pf[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    txh[k] = p.x;
    tyh[k] = p.y;
    txl[k] = p.z;
    tyl[k] = p.w;
  }
#pragma unroll 2
  for (int l = 0; l < nt; ++l) {
    const float4 p = sp[l];
    const float2 q = sq[l];
#pragma unroll
    for (int k = 0; k < kT32; ++k) {
      float cx, cy;
      f32_pair<KIND>(txh[k], tyh[k], txl[k], tyl[k], tnx[k], tny[k], p, q.x, q.y, cx, cy);
      if (DIAG && a0 + k * kB32 == jt + l) cx = cy = 0.0f;  // the self pair (r = 0)
      ax[k] += cx;
      ay[k] += cy;
    }
  }
}

// Far tiles: plain FP32 coordinates relative to the target block's centre.
// Their rounding (|x'| 2^-24 with |x'| at most ~3 |r| for far pairs) is
// below 2e-7 of each term.  The two lanes of the packed FP32x2 instructions
// hold two sources for the same target, read as one 16-byte pair
// (-x'_l, -x'_l+1, -y'_l, -y'_l+1), so that D = T + (-P) = r.  On GB300 the
// FMA pipe retires 128 FP32 lanes a clock per SM whether packed or not, so
// packing halves the issue slots, not the pipe cycles; the loop costs 7 FP32
// lane operations and one MUFU reciprocal a pair.  (Sharing one MUFU operation
// between two reciprocals, 1/a = b rcp(ab), costs 1.5 more FP32 operations a
// pair and measured slower.)
template <int KIND>
__device__ __forceinline__ void tile_far2(const float4* __restrict__ sp2, const float4* __restrict__ sq2, int np,
                                          const float2* TX, const float2* TY, const float2* NX, const float2* NY,
                                          float2* AX, float2* AY) {
#pragma unroll(KIND == 0 ? 4 : 2)
  for (int l = 0; l < np; ++l) {
    const float4 p = sp2[l];
    const float2 px = make_float2(p.x, p.y), py = make_float2(p.z, p.w);
    float2 q1, q2;
    if (KIND == 0) {
      q1 = reinterpret_cast<const float2*>(sq2)[l];
    } else {
      const float4 q = sq2[l];
      q1 = make_float2(q.x, q.y);
      q2 = make_float2(q.z, q.w);
    }
#pragma unroll
    for (int k = 0; k < kT32; ++k) {
      const float2 dx = __fadd2_rn(TX[k], px);
      const float2 dy = __fadd2_rn(TY[k], py);
      const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
      const float2 inv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
      if (KIND == 0) {
        const float2 sc = __fmul2_rn(q1, inv);
        AX[k] = __ffma2_rn(dx, sc, AX[k]);
        AY[k] = __ffma2_rn(dy, sc, AY[k]);
      } else {
        const float2 rq = __ffma2_rn(dx, q1, __fmul2_rn(dy, q2));
        const float2 rn = __ffma2_rn(dx, NX[k], __fmul2_rn(dy, NY[k]));
        const float2 c = __fmul2_rn(__fmul2_rn(rq, rn), __fmul2_rn(inv, inv));
        AX[k] = __ffma2_rn(c, dx, AX[k]);
        AY[k] = __ffma2_rn(c, dy, AY[k]);
      }
    }
  }
}

// s + e += t with the rounding error of the leading sum kept (TwoSum)
__device__ __forceinline__ void comp_add(float& s, float& e, float t) {
  const float u = s + t;
  const float bb = u - s;
  e += (s - (u - bb)) + (t - bb);
  s = u;
}

// Union of the bounding boxes of bodies [b0, b1].
__device__ __forceinline__ float4 body_range_box(const float4* __restrict__ bbox, int b0, int b1) {
  float4 u = bbox[b0];
  for (int i = b0 + 1; i <= b1; ++i) {
    const float4 b = bbox[i];
    u.x = fminf(u.x, b.x);
    u.y = fminf(u.y, b.y);
    u.z = fmaxf(u.z, b.z);
    u.w = fmaxf(u.w, b.w);
  }
  return u;
}

// FP32 source strengths q_b = sscale_b v_b (two per node for Stokes), once per
// operator application: every target block of k_pair32 reads them.
template <int KIND>
__global__ void k_src32(Geo g, VecRef vr, const double* __restrict__ sscale, const int* __restrict__ stop) {
  if (stop && *stop) return;
  const double* __restrict__ v = vr.ptr();
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < g.M; b += gridDim.x * blockDim.x) {
    if (KIND == 0)
      g.qf[b] = (float)(sscale[b] * v[b]);
    else
      reinterpret_cast<float2*>(g.qf)[b] =
          make_float2((float)(sscale[b] * v[2 * b]), (float)(sscale[b] * v[2 * b + 1]));
  }
}

template <int KIND, bool BATCH>
__global__ void __launch_bounds__(kB32, KIND == 0 ? 12 : 10) k_pair32(Geo g, VecRef vr, const double* __restrict__ sscale,
                                                 PairPlan pp, double* __restrict__ partial,
                                                 const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sp[kTile32];  // near: (xh, yh, xl, yl)
  __shared__ float2 sq[kTile32];
  __shared__ float4 sp2[kTile32 / 2];  // far: source pairs (-x', -x', -y', -y')
  __shared__ float4 sq2[kTile32 / 2];  // far: (q1, q1', q2, q2'); Laplace packs (q, q') pairs
  const int M = g.M;
  const int tbase = blockIdx.x * kB32 * kT32;
  const int tend = min(M, tbase + kB32 * kT32);
  if (BATCH && block_stopped(g, tbase, tend)) {
    zero_partials<KIND>(tbase, tend, M, partial);
    return;
  }
  const SrcRange sr = src_range<BATCH>(g, tbase, tend, pp);
  const int j0 = sr.j0, j1 = sr.j1;
  // the target block's box, centre and half-diagonal
  const float4 tb = body_range_box(g.bbox, g.body_of[tbase], g.body_of[tend - 1]);
  const float cx = 0.5f * (tb.x + tb.z), cy = 0.5f * (tb.y + tb.w);
  const float et = 0.5f * sqrtf((tb.z - tb.x) * (tb.z - tb.x) + (tb.w - tb.y) * (tb.w - tb.y));
  const int a0 = tbase + threadIdx.x;
  float tnx[kT32], tny[kT32];
  float2 TX[kT32], TY[kT32], NX[kT32], NY[kT32];
  // compensated FP32 sums over the tiles: value sx + ex
  float sx[kT32], ex[kT32], sy[kT32], ey[kT32];
#pragma unroll
  for (int k = 0; k < kT32; ++k) {
    const int a = a0 + k * kB32;
    float4 p = make_float4(cx, cy, 0.f, 0.f);
    float2 n = make_float2(0.f, 0.f);
    if (a < M) {
      p = g.pf[a];
      if (KIND == 1) n = g.nf[a];
    }
    const float tlx = (p.x - cx) + p.z, tly = (p.y - cy) + p.w;
    tnx[k] = n.x;
    tny[k] = n.y;
    TX[k] = make_float2(tlx, tlx);
    TY[k] = make_float2(tly, tly);
    NX[k] = make_float2(n.x, n.x);
    NY[k] = make_float2(n.y, n.y);
    sx[k] = ex[k] = sy[k] = ey[k] = 0.f;
  }
  // source tiles never cross a body boundary, so a tile's box is its body's
  for (int jt = j0; jt < j1;) {
    const int sb = g.body_of[jt];
    const int nt = min(kTile32, min(j1, g.body_start[sb + 1]) - jt);
    // far when the boxes are at least both half-diagonals apart (block-uniform)
    const float4 sbx = g.bbox[sb];
    const float gx = fmaxf(0.f, fmaxf(sbx.x - tb.z, tb.x - sbx.z));
    const float gy = fmaxf(0.f, fmaxf(sbx.y - tb.w, tb.y - sbx.w));
    const float es = 0.5f * sqrtf((sbx.z - sbx.x) * (sbx.z - sbx.x) + (sbx.w - sbx.y) * (sbx.w - sbx.y));
    const float gap2 = gx * gx + gy * gy;
    const float need = fmaxf(et, es);
    const bool far = gap2 > 0.f && gap2 >= need * need;
    // far tiles are padded to an even count with a zero-strength copy of the last source
    const int ntl = far ? (nt + 1) & ~1 : nt;
    __syncthreads();
    for (int l = threadIdx.x; l < ntl; l += kB32) {
      const int b = jt + min(l, nt - 1);
      const float4 p = g.pf[b];
      float q1 = 0.f, q2 = 0.f;
      if (l < nt) {
        if (KIND == 0) {
          q1 = g.qf[b];
        } else {
          const float2 qq = reinterpret_cast<const float2*>(g.qf)[b];
          q1 = qq.x;
          q2 = qq.y;
        }
      }
      if (far) {
        float* pp = reinterpret_cast<float*>(&sp2[l >> 1]);
        pp[l & 1] = -((p.x - cx) + p.z);
        pp[2 + (l & 1)] = -((p.y - cy) + p.w);
        if (KIND == 0) {
          reinterpret_cast<float*>(sq2)[l] = q1;
        } else {
          float* qq = reinterpret_cast<float*>(&sq2[l >> 1]);
          qq[l & 1] = q1;
          qq[2 + (l & 1)] = q2;
        }
      } else {
        sp[l] = p;
        sq[l] = make_float2(q1, q2);
      }
    }
    __syncthreads();
    float ax[kT32], ay[kT32];
    if (far) {
      float2 AX[kT32], AY[kT32];
#pragma unroll
      for (int k = 0; k < kT32; ++k) AX[k] = AY[k] = make_float2(0.f, 0.f);
      tile_far2<KIND>(sp2, sq2, ntl >> 1, TX, TY, NX, NY, AX, AY);
#pragma unroll
      for (int k = 0; k < kT32; ++k) {
        ax[k] = AX[k].x + AX[k].y;
        ay[k] = AY[k].x + AY[k].y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kT32; ++k) ax[k] = ay[k] = 0.f;
      if ((jt < tend) && (jt + nt > tbase))
        tile_near<KIND, true>(g.pf, sp, sq, nt, jt, a0, M, tnx, tny, ax, ay);
      else
        tile_near<KIND, false>(g.pf, sp, sq, nt, jt, a0, M, tnx, tny, ax, ay);
    }
    if (BATCH) {
      // batched solves: a tile counts only for its own problem's targets (a block
      // may straddle two problems)
#pragma unroll
      for (int k = 0; k < kT32; ++k)
        if (!same_problem(g, a0 + k * kB32, jt)) ax[k] = ay[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kT32; ++k) {
      comp_add(sx[k], ex[k], ax[k]);
      comp_add(sy[k], ey[k], ay[k]);
    }
    jt += nt;
  }
#pragma unroll
  for (int k = 0; k < kT32; ++k) {
    const int a = a0 + k * kB32;
    if (a < M) {
      if (KIND == 0) {
        // n_a . (sx + ex, sy + ey) in float-float: the normal's hi/lo split,
        // error-free products, one TwoSum (no FP64 pipe per target and block)
        const float4 n = g.nff[a];
        float p1, e1, p2, e2, h, l;
        ff_mul(n.x, n.y, sx[k], ex[k], p1, e1);
        ff_mul(n.z, n.w, sy[k], ey[k], p2, e2);
        two_sum(p1, p2, h, l);
        reinterpret_cast<float2*>(partial)[(long long)blockIdx.y * M + a] = make_float2(h, l + (e1 + e2));
      } else {
        // (sx + ex, sy + ey) as two float-float pairs: no FP64 pipe in the kernel
        float hx, lx, hy, ly;
        two_sum(sx[k], ex[k], hx, lx);
        two_sum(sy[k], ey[k], hy, ly);
        reinterpret_cast<float4*>(partial)[(long long)blockIdx.y * M + a] = make_float4(hx, lx, hy, ly);
      }
    }
  }
}

// ------------------------------------------------------- symmetric FP32 ----
// Laplace pair sums with each reciprocal used for both directions of a pair.
// The M nodes are cut into tiles of kTS = 256 consecutive nodes; one CTA takes
// one unordered pair of tiles (A = tile i, B = tile j, i <= j) and writes the
// contribution of B's sources to A's targets into partial[j][A] and that of
// A's sources to B's targets into partial[i][B]: every (source tile, target
// tile) slot is written exactly once, and the epilogue adds the S = tiles
// slots of a target in a fixed order (deterministic).
//
// Far tile pairs (boxes at least both half-diagonals apart): with r = x_a - x_b
// and w = 1/|r|^2, target a gains q_b r w and target b gains -q_a r w, so one
// MUFU reciprocal and about 10 FP32 lane operations serve two directed pairs
// (the directed kernel: one reciprocal and 7 operations for one).  Each lane
// holds four A targets in registers (packed two by two); B's sources sit in
// shared memory and are visited on a diagonal schedule (lane l takes source
// (l + k) mod 32 of the current group of 32 at step k), and the accumulator of
// B's source travels with it from lane to lane by a warp shuffle, so no two
// lanes ever add into the same place.  Coordinates are relative to A's box
// centre, as in the directed far tiles.  Near tile pairs (and i = j) run the
// directed near path in both directions (exact hi/lo differences).
constexpr int kTS = kB32 * kT32;  // 256 nodes a tile

__device__ __forceinline__ void tri_decode(int t, int& i, int& j) {
  int jj = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);  // then corrected exactly
  while ((long long)(jj + 1) * (jj + 2) / 2 <= t) ++jj;
  while ((long long)jj * (jj + 1) / 2 > t) --jj;
  j = jj;
  i = t - jj * (jj + 1) / 2;
}

// Is box b far from box a (gap at least both half-diagonals)?
__device__ __forceinline__ bool boxes_far(float4 a, float4 b) {
  const float gx = fmaxf(0.f, fmaxf(b.x - a.z, a.x - b.z));
  const float gy = fmaxf(0.f, fmaxf(b.y - a.w, a.y - b.w));
  const float ea = 0.5f * sqrtf((a.z - a.x) * (a.z - a.x) + (a.w - a.y) * (a.w - a.y));
  const float eb = 0.5f * sqrtf((b.z - b.x) * (b.z - b.x) + (b.w - b.y) * (b.w - b.y));
  const float gap2 = gx * gx + gy * gy;
  const float need = fmaxf(ea, eb);
  return gap2 > 0.f && gap2 >= need * need;
}

// partial[slot][a] = n_a . (ax, ay) in float-float (the normal's hi/lo split),
// stored as the float pair (h, l): no FP64 pipe in the kernel
__device__ __forceinline__ void write_projected(const Geo& g, int a, int slot, float ax, float ay,
                                                double* __restrict__ partial) {
  const float4 n = g.nff[a];
  float p1, e1, p2, e2, h, l;
  ff_mul(n.x, n.y, ax, 0.f, p1, e1);
  ff_mul(n.z, n.w, ay, 0.f, p2, e2);
  two_sum(p1, p2, h, l);
  reinterpret_cast<float2*>(partial)[(long long)slot * g.M + a] = make_float2(h, l + (e1 + e2));
}

// Directed near pass: targets [t0, t0 + kTS) gain the sources [s0, s1) (one
// tile, exact hi/lo differences), written to partial[slot].
template <bool DIAG>
__device__ __forceinline__ void sym_near_pass(const Geo& g, int t0, int s0, int s1, int slot,
                                              double* __restrict__ partial, float4* sp, float2* sq) {
  const int M = g.M, nt = s1 - s0;
  __syncthreads();  // the tile buffers may still be read
  for (int l = threadIdx.x; l < nt; l += kB32) {
    sp[l] = g.pf[s0 + l];
    sq[l] = make_float2(g.qf[s0 + l], 0.f);
  }
  __syncthreads();
  float ax[kT32], ay[kT32], tnx[kT32], tny[kT32];
#pragma unroll
  for (int k = 0; k < kT32; ++k) ax[k] = ay[k] = tnx[k] = tny[k] = 0.f;
  tile_near<0, DIAG>(g.pf, sp, sq, nt, s0, t0 + threadIdx.x, M, tnx, tny, ax, ay);
#pragma unroll
  for (int k = 0; k < kT32; ++k) {
    const int a = t0 + threadIdx.x + k * kB32;
    if (a < M) write_projected(g, a, slot, ax[k], ay[k], partial);
  }
}

__global__ void __launch_bounds__(kB32, 12) k_pair32s(Geo g, int ntile, double* __restrict__ partial,
                                                      const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ __align__(16) unsigned char sm_raw[kTS * 32];  // far: sources + 2 accumulator rows; near: sp, sq
  const int M = g.M;
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  const int A0 = ti * kTS, A1 = min(M, A0 + kTS), B0 = tj * kTS, B1 = min(M, B0 + kTS);
  const float4 boxA = body_range_box(g.bbox, g.body_of[A0], g.body_of[A1 - 1]);
  const float4 boxB = body_range_box(g.bbox, g.body_of[B0], g.body_of[B1 - 1]);
  if (ti == tj || !boxes_far(boxA, boxB)) {
    float4* sp = reinterpret_cast<float4*>(sm_raw);
    float2* sq = reinterpret_cast<float2*>(sm_raw + kTS * sizeof(float4));
    if (ti == tj) {
      sym_near_pass<true>(g, A0, B0, B1, tj, partial, sp, sq);
    } else {
      sym_near_pass<false>(g, A0, B0, B1, tj, partial, sp, sq);
      sym_near_pass<false>(g, B0, A0, A1, ti, partial, sp, sq);
    }
    return;
  }
  float4* sB = reinterpret_cast<float4*>(sm_raw);                    // (-x', -y', q, 0) per source
  float2* accB = reinterpret_cast<float2*>(sm_raw + kTS * sizeof(float4));  // [2 warps][kTS]
  const float cx = 0.5f * (boxA.x + boxA.z), cy = 0.5f * (boxA.y + boxA.w);
  constexpr float kAway = 1e15f;  // padding: far from everything, zero strength
  for (int l = threadIdx.x; l < kTS; l += kB32) {
    const int b = B0 + l;
    float4 v = make_float4(-kAway, -kAway, 0.f, 0.f);
    if (b < M) {
      const float4 p = g.pf[b];
      v = make_float4(-((p.x - cx) + p.z), -((p.y - cy) + p.w), g.qf[b], 0.f);
    }
    sB[l] = v;
  }
  // four A targets per lane, packed two by two: (t0, t1) and (t2, t3)
  float tx[kT32], ty[kT32], qa[kT32];
#pragma unroll
  for (int k = 0; k < kT32; ++k) {
    const int a = A0 + threadIdx.x + k * kB32;
    tx[k] = ty[k] = kAway;
    qa[k] = 0.f;
    if (a < M) {
      const float4 p = g.pf[a];
      tx[k] = (p.x - cx) + p.z;
      ty[k] = (p.y - cy) + p.w;
      qa[k] = g.qf[a];
    }
  }
  const float2 TXa = make_float2(tx[0], tx[1]), TXb = make_float2(tx[2], tx[3]);
  const float2 TYa = make_float2(ty[0], ty[1]), TYb = make_float2(ty[2], ty[3]);
  const float2 QAa = make_float2(qa[0], qa[1]), QAb = make_float2(qa[2], qa[3]);
  float2 AXa = make_float2(0.f, 0.f), AXb = AXa, AYa = AXa, AYb = AXa;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r0 = 0; r0 < kTS; r0 += 32) {
    float bx = 0.f, by = 0.f;  // accumulator of the source this lane holds (travels)
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float4 src = sB[r0 + ((lane + k) & 31)];
      const float2 sx = make_float2(src.x, src.x), sy = make_float2(src.y, src.y);
      const float2 dxa = __fadd2_rn(TXa, sx), dxb = __fadd2_rn(TXb, sx);
      const float2 dya = __fadd2_rn(TYa, sy), dyb = __fadd2_rn(TYb, sy);
      const float2 r2a = __ffma2_rn(dxa, dxa, __fmul2_rn(dya, dya));
      const float2 r2b = __ffma2_rn(dxb, dxb, __fmul2_rn(dyb, dyb));
      const float2 ia = make_float2(rcp_approx(r2a.x), rcp_approx(r2a.y));
      const float2 ib = make_float2(rcp_approx(r2b.x), rcp_approx(r2b.y));
      const float2 qb = make_float2(src.z, src.z);
      const float2 sba = __fmul2_rn(qb, ia), sbb = __fmul2_rn(qb, ib);
      AXa = __ffma2_rn(dxa, sba, AXa);
      AXb = __ffma2_rn(dxb, sbb, AXb);
      AYa = __ffma2_rn(dya, sba, AYa);
      AYb = __ffma2_rn(dyb, sbb, AYb);
      const float2 saa = __fmul2_rn(QAa, ia), sab = __fmul2_rn(QAb, ib);
      const float2 ux = __ffma2_rn(dxb, sab, __fmul2_rn(dxa, saa));
      const float2 uy = __ffma2_rn(dyb, sab, __fmul2_rn(dya, saa));
      bx -= ux.x + ux.y;  // the source gains -q_a r w
      by -= uy.x + uy.y;
      // hand the accumulator to the lane that takes this source next
      bx = __shfl_sync(0xffffffffu, bx, (lane + 1) & 31);
      by = __shfl_sync(0xffffffffu, by, (lane + 1) & 31);
    }
    accB[warp * kTS + r0 + lane] = make_float2(bx, by);  // back at its own lane: source r0 + lane
  }
  {
    const int a = A0 + threadIdx.x;
    if (a < M) write_projected(g, a, tj, AXa.x, AYa.x, partial);
    if (a + kB32 < M) write_projected(g, a + kB32, tj, AXa.y, AYa.y, partial);
    if (a + 2 * kB32 < M) write_projected(g, a + 2 * kB32, tj, AXb.x, AYb.x, partial);
    if (a + 3 * kB32 < M) write_projected(g, a + 3 * kB32, tj, AXb.y, AYb.y, partial);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < kTS; l += kB32) {
    const int b = B0 + l;
    if (b < M) {
      const float2 u = accB[l], v = accB[kTS + l];
      write_projected(g, b, ti, u.x + v.x, u.y + v.y, partial);
    }
  }
}

// ------------------------------------------------------------ float-float ----
// Pair sums in float-float ("double-single") arithmetic on the FP32 pipes, for
// residuals that must be accurate far beyond FP32: every quantity is an
// unevaluated sum h + l of two floats (about 48 significant bits).
//  - positions: exact split x = h + m + l (quanta from g.qscale, computed
//    once per geometry), so that dx = (h_a - h_b) + (m_a - m_b) + (l_a - l_b)
//    has exact leading parts for every pair, near or far;
//  - products: error-free a*b = p + fma(a, b, -p);
//  - reciprocal: MUFU rcp.approx seed y0 refined by one Newton step in
//    float-float, 1/r2 = y0 + y0 (1 - r2 y0);
//  - sums: TwoSum (Knuth) for the leading parts, trailing parts added, within
//    a tile and across tiles (no FP64 in the loop: GB300's FP64 pipe is slow).
constexpr int kBF = 64, kTF = 4, kTileF = 256;

template <int KIND, bool DIAG>
__device__ __forceinline__ void tile_ff(const float4* __restrict__ sa, const float2* __restrict__ sb,
                                        const float4* __restrict__ sq, int nt, int jt, int a0, const FFTarget* t,
                                        float* axh, float* axl, float* ayh, float* ayl) {
  for (int l = 0; l < nt; ++l) {
    const float4 pa = sa[l];  // (xh, xm, yh, ym)
    const float2 pb = sb[l];  // (xl, yl)
    const float4 q = sq[l];   // (q1h, q1l, q2h, q2l)
#pragma unroll
    for (int k = 0; k < kTF; ++k) {
      float cxh, cxl, cyh, cyl;
      ff_pair<KIND>(t[k], pa, pb, q, cxh, cxl, cyh, cyl);
      if (DIAG && a0 + k * kBF == jt + l) cxh = cxl = cyh = cyl = 0.0f;  // the self pair
      ff_acc(axh[k], axl[k], cxh, cxl);
      ff_acc(ayh[k], ayl[k], cyh, cyl);
    }
  }
}

template <int KIND, bool BATCH>
__global__ void __launch_bounds__(kBF) k_pair_ff(Geo g, VecRef vr, const double* __restrict__ sscale, PairPlan pp,
                                                 double* __restrict__ partial, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sa[kTileF];
  __shared__ float2 sb[kTileF];
  __shared__ float4 sq[kTileF];
  const double* __restrict__ v = vr.ptr();
  const int M = g.M;
  const int tbase = blockIdx.x * kBF * kTF;
  const int tend = min(M, tbase + kBF * kTF);
  if (BATCH && block_stopped(g, tbase, tend)) {
    zero_partials<KIND>(tbase, tend, M, partial);
    return;
  }
  const int a0 = tbase + threadIdx.x;
  const SrcRange sr = src_range<BATCH>(g, tbase, tend, pp);
  const int j0 = sr.j0, j1 = sr.j1;
  FFTarget t[kTF];
  // float-float sums over the tiles
  float sxh[kTF], sxl[kTF], syh[kTF], syl[kTF];
#pragma unroll
  for (int k = 0; k < kTF; ++k) {
    const int a = a0 + k * kBF;
    const float4 p = a < M ? g.xff[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 pl = a < M ? g.xfl[a] : make_float2(0.f, 0.f);
    t[k].xh = p.x;
    t[k].xm = p.y;
    t[k].yh = p.z;
    t[k].ym = p.w;
    t[k].xl = pl.x;
    t[k].yl = pl.y;
    t[k].n = (KIND == 1 && a < M) ? g.nff[a] : make_float4(0.f, 0.f, 0.f, 0.f);
    sxh[k] = sxl[k] = syh[k] = syl[k] = 0.f;
  }
  for (int jt = j0; jt < j1;) {
    const int nt = tile_len<BATCH>(g, jt, min(kTileF, j1 - jt));
    __syncthreads();
    for (int l = threadIdx.x; l < nt; l += kBF) {
      const int b = jt + l;
      sa[l] = g.xff[b];
      sb[l] = g.xfl[b];
      const double q1 = KIND == 0 ? sscale[b] * v[b] : sscale[b] * v[2 * b];
      const double q2 = KIND == 0 ? 0.0 : sscale[b] * v[2 * b + 1];
      const float q1h = (float)q1, q2h = (float)q2;
      sq[l] = make_float4(q1h, (float)(q1 - (double)q1h), q2h, (float)(q2 - (double)q2h));
    }
    __syncthreads();
    float axh[kTF], axl[kTF], ayh[kTF], ayl[kTF];
#pragma unroll
    for (int k = 0; k < kTF; ++k) axh[k] = axl[k] = ayh[k] = ayl[k] = 0.f;
    if ((jt < tend) && (jt + nt > tbase))
      tile_ff<KIND, true>(sa, sb, sq, nt, jt, a0, t, axh, axl, ayh, ayl);
    else
      tile_ff<KIND, false>(sa, sb, sq, nt, jt, a0, t, axh, axl, ayh, ayl);
    if (BATCH) {
#pragma unroll
      for (int k = 0; k < kTF; ++k)
        if (!same_problem(g, a0 + k * kBF, jt)) axh[k] = axl[k] = ayh[k] = ayl[k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kTF; ++k) {
      ff_acc(sxh[k], sxl[k], axh[k], axl[k]);
      ff_acc(syh[k], syl[k], ayh[k], ayl[k]);
    }
    jt += nt;
  }
#pragma unroll
  for (int k = 0; k < kTF; ++k) {
    const int a = a0 + k * kBF;
    const double dax = (double)sxh[k] + (double)sxl[k], day = (double)syh[k] + (double)syl[k];
    if (a < M) {
      if (KIND == 0)
        partial[(long long)blockIdx.y * M + a] = g.nx[a] * dax + g.ny[a] * day;
      else {
        partial[((long long)blockIdx.y * M + a) * 2] = dax;
        partial[((long long)blockIdx.y * M + a) * 2 + 1] = day;
      }
    }
  }
}

// ------------------------------------------------- symmetric float-float ----
// The float-float Laplace pair sum on unordered pairs of 256-node tiles, each
// reciprocal (MUFU seed + one float-float Newton step) and each difference and
// |r|^2 serving both directions: target a gains q_b r w, target b gains
// -q_a r w.  Float-float positions give exact leading differences for every
// pair, so every pair of different tiles takes the symmetric loop; a tile
// with itself (the self pairs) runs the directed float-float pass.  The
// source's float-float accumulator travels between lanes by warp shuffle on
// the diagonal schedule of k_pair32s.  Partials: FP64, one slot per (source
// tile, target tile), projected on the target normal in FP64.
constexpr int kTFS = 2;                      // targets a lane
constexpr int kBFS = kTileF / kTFS;          // 128 threads a CTA

// Packed forms of the float-float helpers: the two halves of a float2 are two
// independent values, each rounded exactly as the scalar form rounds it.
__device__ __forceinline__ float2 neg2f(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void ff_mul2(float2 ah, float2 al, float2 bh, float2 bl, float2& p, float2& e) {
  p = __fmul2_rn(ah, bh);
  e = __ffma2_rn(ah, bh, neg2f(p));
  e = __ffma2_rn(ah, bl, __ffma2_rn(al, bh, e));
}
__device__ __forceinline__ void ff_acc2(float2& sh, float2& sl, float2 th, float2 tl) {
  const float2 u = __fadd2_rn(sh, th);
  const float2 bb = __fadd2_rn(u, neg2f(sh));
  const float2 e = __fadd2_rn(__fadd2_rn(sh, neg2f(__fadd2_rn(u, neg2f(bb)))), __fadd2_rn(th, neg2f(bb)));
  sh = u;
  sl = __fadd2_rn(sl, __fadd2_rn(e, tl));
}

__device__ __forceinline__ void ff_write_projected(const Geo& g, int a, int slot, float xh, float xl, float yh,
                                                   float yl, double* __restrict__ partial) {
  const double dax = (double)xh + (double)xl, day = (double)yh + (double)yl;
  partial[(long long)slot * g.M + a] = g.nx[a] * dax + g.ny[a] * day;
}

__global__ void __launch_bounds__(kBFS, 6) k_pair_ffs(Geo g, int ntile, double* __restrict__ partial,
                                                     const double* __restrict__ sscale, VecRef vr,
                                                     const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float4 sA[kTileF];  // (xh, xm, yh, ym)
  __shared__ float4 sC[kTileF];  // (xl, yl, qh, ql)
  __shared__ float4 accB[kBFS / 32][kTileF];  // per warp: the sources' (xh, xl, yh, yl)
  const double* __restrict__ v = vr.ptr();
  const int M = g.M;
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  const int A0 = ti * kTileF, B0 = tj * kTileF;
  if (ti == tj) {
    // directed float-float pass of the tile with itself (excludes r = 0)
    const int a1 = min(M, A0 + kTileF), nt = a1 - A0;
    for (int l = threadIdx.x; l < nt; l += kBFS) {
      const int b = A0 + l;
      const float4 xa = g.xff[b];
      const float2 xl = g.xfl[b];
      const double q = sscale[b] * v[b];
      const float qh = (float)q;
      sA[l] = xa;
      sC[l] = make_float4(xl.x, xl.y, qh, (float)(q - (double)qh));
    }
    __syncthreads();
    for (int m = 0; m < kTFS; ++m) {
      const int a = A0 + threadIdx.x + m * kBFS;
      if (a >= M) continue;
      FFTarget t;
      const float4 p = g.xff[a];
      const float2 pl = g.xfl[a];
      t.xh = p.x; t.xm = p.y; t.yh = p.z; t.ym = p.w; t.xl = pl.x; t.yl = pl.y;
      t.n = make_float4(0.f, 0.f, 0.f, 0.f);
      float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f;
      for (int l = 0; l < nt; ++l) {
        if (A0 + l == a) continue;
        const float4 c = sC[l];
        float cxh, cxl, cyh, cyl;
        ff_pair<0>(t, sA[l], make_float2(c.x, c.y), make_float4(c.z, c.w, 0.f, 0.f), cxh, cxl, cyh, cyl);
        ff_acc(axh, axl, cxh, cxl);
        ff_acc(ayh, ayl, cyh, cyl);
      }
      ff_write_projected(g, a, ti, axh, axl, ayh, ayl, partial);
    }
    return;
  }
  // sources of tile B, negated (so that a difference is a packed add);
  // padding far from everything with zero strength
  for (int l = threadIdx.x; l < kTileF; l += kBFS) {
    const int b = B0 + l;
    float4 xa = make_float4(-1e15f, 0.f, -1e15f, 0.f), c = make_float4(0.f, 0.f, 0.f, 0.f);
    if (b < M) {
      const float4 x = g.xff[b];
      const float2 xl = g.xfl[b];
      const double q = sscale[b] * v[b];
      const float qh = (float)q;
      xa = make_float4(-x.x, -x.y, -x.z, -x.w);
      c = make_float4(-xl.x, -xl.y, qh, (float)(q - (double)qh));
    }
    sA[l] = xa;
    sC[l] = c;
  }
  // the kTFS = 2 targets of tile A a lane, packed as the two halves of
  // FP32x2 operands (all of tile A is inside [0, M): ti < tj)
  static_assert(kTFS == 2, "two targets a lane, one packed pair");
  float2 TXH, TXM, TXL, TYH, TYM, TYL, QAH, QAL;
  {
    const int a0 = A0 + threadIdx.x, a1 = a0 + kBFS;
    const float4 p0 = g.xff[a0], p1 = g.xff[a1];
    const float2 l0 = g.xfl[a0], l1 = g.xfl[a1];
    TXH = make_float2(p0.x, p1.x);
    TXM = make_float2(p0.y, p1.y);
    TYH = make_float2(p0.z, p1.z);
    TYM = make_float2(p0.w, p1.w);
    TXL = make_float2(l0.x, l1.x);
    TYL = make_float2(l0.y, l1.y);
    const double q0 = sscale[a0] * v[a0], q1 = sscale[a1] * v[a1];
    const float h0 = (float)q0, h1 = (float)q1;
    QAH = make_float2(h0, h1);
    QAL = make_float2((float)(q0 - (double)h0), (float)(q1 - (double)h1));
  }
  float2 AXH = make_float2(0.f, 0.f), AXL = AXH, AYH = AXH, AYL = AXH;
  const float2 ONE = make_float2(1.f, 1.f), TWO = make_float2(2.f, 2.f);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r0 = 0; r0 < kTileF; r0 += 32) {
    float bxh = 0.f, bxl = 0.f, byh = 0.f, byl = 0.f;  // travels with its source
#pragma unroll 2
    for (int k = 0; k < 32; ++k) {
      const int l = r0 + ((lane + k) & 31);
      const float4 sa = sA[l], sc = sC[l];
      // float-float differences r = x_a - x_b from the exact splits (as ff_diff)
      const float2 d1x = __fadd2_rn(TXH, make_float2(sa.x, sa.x)), d2x = __fadd2_rn(TXM, make_float2(sa.y, sa.y));
      const float2 d1y = __fadd2_rn(TYH, make_float2(sa.z, sa.z)), d2y = __fadd2_rn(TYM, make_float2(sa.w, sa.w));
      const float2 DXH = __fadd2_rn(d1x, d2x), DYH = __fadd2_rn(d1y, d2y);
      const float2 DXL = __fadd2_rn(__fadd2_rn(d2x, neg2f(__fadd2_rn(DXH, neg2f(d1x)))),
                                    __fadd2_rn(TXL, make_float2(sc.x, sc.x)));
      const float2 DYL = __fadd2_rn(__fadd2_rn(d2y, neg2f(__fadd2_rn(DYH, neg2f(d1y)))),
                                    __fadd2_rn(TYL, make_float2(sc.y, sc.y)));
      // |r|^2 in float-float: error-free squares, an error-free sum of the two,
      // the cross terms, renormalised (as the directed pair)
      const float2 P1 = __fmul2_rn(DXH, DXH), P1E = __ffma2_rn(DXH, DXH, neg2f(P1));
      const float2 P2 = __fmul2_rn(DYH, DYH), P2E = __ffma2_rn(DYH, DYH, neg2f(P2));
      const float2 S = __fadd2_rn(P1, P2);
      const float2 BB = __fadd2_rn(S, neg2f(P1));
      const float2 SE = __fadd2_rn(__fadd2_rn(P1, neg2f(__fadd2_rn(S, neg2f(BB)))), __fadd2_rn(P2, neg2f(BB)));
      const float2 LO = __ffma2_rn(TWO, __ffma2_rn(DXH, DXL, __fmul2_rn(DYH, DYL)),
                                   __fadd2_rn(__fadd2_rn(SE, P1E), P2E));
      const float2 R2H = __fadd2_rn(S, LO);
      const float2 R2L = __fadd2_rn(LO, neg2f(__fadd2_rn(R2H, neg2f(S))));
      // 1/|r|^2: MUFU seed and one float-float Newton step
      const float2 Y0 = make_float2(rcp_approx(R2H.x), rcp_approx(R2H.y));
      const float2 EE = __ffma2_rn(neg2f(R2L), Y0, __ffma2_rn(neg2f(R2H), Y0, ONE));
      const float2 IL = __fmul2_rn(Y0, EE);
      // target a gains q_b r w
      float2 CH, CL, PH, PL;
      ff_mul2(make_float2(sc.z, sc.z), make_float2(sc.w, sc.w), Y0, IL, CH, CL);
      ff_mul2(CH, CL, DXH, DXL, PH, PL);
      ff_acc2(AXH, AXL, PH, PL);
      ff_mul2(CH, CL, DYH, DYL, PH, PL);
      ff_acc2(AYH, AYL, PH, PL);
      // the source gains -q_a r w (both targets' terms, in the order of the
      // scalar pass: target 0, then target 1)
      ff_mul2(QAH, QAL, Y0, IL, CH, CL);
      ff_mul2(CH, CL, DXH, DXL, PH, PL);
      ff_acc(bxh, bxl, -PH.x, -PL.x);
      ff_acc(bxh, bxl, -PH.y, -PL.y);
      ff_mul2(CH, CL, DYH, DYL, PH, PL);
      ff_acc(byh, byl, -PH.x, -PL.x);
      ff_acc(byh, byl, -PH.y, -PL.y);
      const int nxt = (lane + 1) & 31;
      bxh = __shfl_sync(0xffffffffu, bxh, nxt);
      bxl = __shfl_sync(0xffffffffu, bxl, nxt);
      byh = __shfl_sync(0xffffffffu, byh, nxt);
      byl = __shfl_sync(0xffffffffu, byl, nxt);
    }
    accB[warp][r0 + lane] = make_float4(bxh, bxl, byh, byl);
  }
  ff_write_projected(g, A0 + threadIdx.x, tj, AXH.x, AXL.x, AYH.x, AYL.x, partial);
  ff_write_projected(g, A0 + threadIdx.x + kBFS, tj, AXH.y, AXL.y, AYH.y, AYL.y, partial);
  __syncthreads();
  for (int l = threadIdx.x; l < kTileF; l += kBFS) {
    const int b = B0 + l;
    if (b >= M) continue;
    // the warps' sums in a fixed order
    float4 t = accB[0][l];
#pragma unroll
    for (int w = 1; w < kBFS / 32; ++w) {
      const float4 u = accB[w][l];
      ff_acc(t.x, t.y, u.x, u.y);
      ff_acc(t.z, t.w, u.z, u.w);
    }
    ff_write_projected(g, b, ti, t.x, t.y, t.z, t.w, partial);
  }
}

// --------------------------------------------------------------- epilogue ----
constexpr int kBE = 256;

// One block per body: completion moments, then per node
//   y = Kv (constant applied) + diagonal limit + [L]; out = sign (1/2 v + oscale y).
// (sh, sl) += (h, l) in float-float
__device__ __forceinline__ void ffadd(float& sh, float& sl, float h, float l) {
  float u, e;
  two_sum(sh, h, u, e);
  sh = u;
  sl += e + l;
}

template <int KIND, int B>
__global__ void __launch_bounds__(B) k_epilogue(Geo g, VecRef vr, const double* __restrict__ partial,
                                                  int S, int scaled, int with_L, double alpha, double sign,
                                                  VecRef outr, const int* __restrict__ stop, int pff) {
  if (stop && *stop) return;
  __shared__ double sh[B / 32];
  const double* __restrict__ v = vr.ptr();
  double* __restrict__ out = outr.ptr();
  const int M = g.M;
  const int i = blockIdx.x;
  const int a0 = g.body_start[i], a1 = g.body_start[i + 1];
  const double xc = g.xc[i], yc = g.yc[i];
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  __shared__ double cfs[2];  // completion weights alpha/|Gamma_i|, alpha/W_i: one FP64 division each per block
  if (with_L && alpha > 0.0 && threadIdx.x == 0) {
    cfs[0] = alpha / g.len[i];
    cfs[1] = KIND == 1 ? alpha / g.W[i] : 1.0;
  }
  if (with_L) {
    for (int a = a0 + threadIdx.x; a < a1; a += B) {
      const double s = scaled ? g.sw[a] : g.w[a];
      if (KIND == 0) {
        m0 += s * v[a];
      } else {
        const double f1 = s * v[2 * a], f2 = s * v[2 * a + 1];
        m0 += f1;
        m1 += f2;
        m2 += -(g.y[a] - yc) * f1 + (g.x[a] - xc) * f2;
      }
    }
    m0 = block_sum<B>(m0, sh);
    if (KIND == 1) {
      m1 = block_sum<B>(m1, sh);
      m2 = block_sum<B>(m2, sh);
    }
    if (alpha > 0.0) {  // completion weighted per body: force part alpha/|Gamma_i|, torque part alpha/W_i
      const double cf = cfs[0];  // written before block_sum's barriers
      m0 *= cf;
      m1 *= cf;
      if (KIND == 1) m2 *= cfs[1];
    }
  }
  for (int a = a0 + threadIdx.x; a < a1; a += B) {
    const double os = scaled ? g.sw[a] : 1.0;
    const double wk = g.w[a] * g.kappa[a];
    if (KIND == 0) {
      double k;
      if (pff) {
        // float-float partials of the FP32 pair sums: two independent float-float
        // sums (loads in flight), added in a fixed order, converted once
        const float2* __restrict__ pf2 = reinterpret_cast<const float2*>(partial);
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        int s = 0;
        for (; s + 2 <= S; s += 2) {
          const float2 u = pf2[(long long)s * M + a], v = pf2[(long long)(s + 1) * M + a];
          ffadd(h0, l0, u.x, u.y);
          ffadd(h1, l1, v.x, v.y);
        }
        if (s < S) {
          const float2 u = pf2[(long long)s * M + a];
          ffadd(h0, l0, u.x, u.y);
        }
        ffadd(h0, l0, h1, l1);
        k = (double)h0 + (double)l0;
      } else {
        // four independent sums over the source splits (loads in flight), added in a fixed order
        double k0 = 0.0, k1 = 0.0, k2 = 0.0, k3 = 0.0;
        int s = 0;
        for (; s + 4 <= S; s += 4) {
          k0 += partial[(long long)s * M + a];
          k1 += partial[(long long)(s + 1) * M + a];
          k2 += partial[(long long)(s + 2) * M + a];
          k3 += partial[(long long)(s + 3) * M + a];
        }
        for (; s < S; ++s) k0 += partial[(long long)s * M + a];
        k = (k0 + k1) + (k2 + k3);
      }
      // os y with y = -k/2pi - wk mu/4pi + m0 and mu = v/os: the diagonal term
      // os wk mu/4pi = wk v/4pi needs no division
      out[a] = sign * (0.5 * v[a] + os * (m0 - kInv2Pi * k) - kInv4Pi * wk * v[a]);
    } else {
      double k1 = 0.0, k2 = 0.0;
      if (pff) {
        const float4* __restrict__ pf4 = reinterpret_cast<const float4*>(partial);
        float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int s = 0; s < S; ++s) {
          const float4 u = pf4[(long long)s * M + a];
          ffadd(h1, l1, u.x, u.y);
          ffadd(h2, l2, u.z, u.w);
        }
        k1 = (double)h1 + (double)l1;
        k2 = (double)h2 + (double)l2;
      } else {
        double k1b = 0.0, k2b = 0.0;
        int s = 0;
        for (; s + 2 <= S; s += 2) {
          const double2 p0 = reinterpret_cast<const double2*>(partial)[(long long)s * M + a];
          const double2 p1 = reinterpret_cast<const double2*>(partial)[(long long)(s + 1) * M + a];
          k1 += p0.x;
          k2 += p0.y;
          k1b += p1.x;
          k2b += p1.y;
        }
        if (s < S) {
          const double2 p0 = reinterpret_cast<const double2*>(partial)[(long long)s * M + a];
          k1 += p0.x;
          k2 += p0.y;
        }
        k1 += k1b;
        k2 += k2b;
      }
      // os y with the diagonal term os dd t, dd = -wk (t . mu)/2pi and mu = v/os:
      // os dd = -wk (t . v)/2pi needs no division
      const double tx = -g.ny[a], ty = g.nx[a];
      const double v1 = v[2 * a], v2 = v[2 * a + 1];
      const double odd = -0.5 * kInvPi * wk * (tx * v1 + ty * v2);
      const double px = -(g.y[a] - yc), py = g.x[a] - xc;
      out[2 * a] = sign * (0.5 * v1 + os * (m0 + px * m2 - kInvPi * k1) + odd * tx);
      out[2 * a + 1] = sign * (0.5 * v2 + os * (m1 + py * m2 - kInvPi * k2) + odd * ty);
    }
  }
}

// The epilogue of the FP32 operator (the inner solves).  On GB300 most of
// k_epilogue's FP64-pipe time goes to the per-body completion moments and
// their block sums; here they run on the FP32 pipe in float-float (FP32
// products s v with their exact rounding errors, error-free sums), which
// keeps them accurate well beyond FP32 (the per-term roundings of s and v
// average out; no total is ever rounded to FP32), and the per-node output
// is k_epilogue's FP64 expression.  Fixed order throughout (deterministic).
// (h, l) += (bh, bl) in float-float
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

// (h, l) += a b with the product's rounding error
__device__ __forceinline__ void ff_add_prod(float& h, float& l, float a, float b) {
  const float p = a * b;
  ff_add(h, l, p, fmaf(a, b, -p));
}

// Block sum of a float-float value; the result, as a double, in *out (shared)
// after the call.  sh needs B/32 float2.
template <int B>
__device__ __forceinline__ void block_sum_ff(float h, float l, float2* sh, double* out) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
    ff_add(h, l, oh, ol);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(h, l);
  __syncthreads();
  if (threadIdx.x == 0) {
    float th = sh[0].x, tl = sh[0].y;
#pragma unroll
    for (int k = 1; k < B / 32; ++k) ff_add(th, tl, sh[k].x, sh[k].y);
    *out = (double)th + (double)tl;
  }
}

template <int KIND, int B>
__global__ void __launch_bounds__(B) k_epilogue32(Geo g, VecRef vr, const double* __restrict__ partial, int S,
                                                    int scaled, int with_L, double alpha, double sign, VecRef outr,
                                                    const int* __restrict__ stop, int pff) {
  if (stop && *stop) return;
  __shared__ float2 sh[B / 32];
  __shared__ float cst[4];   // body centre split hi + lo
  __shared__ double mom[3];  // completion moments, weighted
  const double* __restrict__ v = vr.ptr();
  double* __restrict__ out = outr.ptr();
  const int M = g.M;
  const int i = blockIdx.x;
  const int a0 = g.body_start[i], a1 = g.body_start[i + 1];
  const double xc = g.xc[i], yc = g.yc[i];
  if (threadIdx.x == 0) {
    const float hx = (float)xc, hy = (float)yc;
    cst[0] = hx;
    cst[1] = hy;
    cst[2] = (float)(xc - (double)hx);
    cst[3] = (float)(yc - (double)hy);
    mom[0] = mom[1] = mom[2] = 0.0;
  }
  __syncthreads();
  if (with_L) {
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
    for (int a = a0 + threadIdx.x; a < a1; a += B) {
      const float2 wk = g.wkf[a];
      const float sc = scaled ? wk.x : wk.x * wk.x;
      if (KIND == 0) {
        ff_add_prod(h0, l0, sc, (float)v[a]);
      } else {
        const float4 P = g.pf[a];
        const float dx = (P.x - cst[0]) + (P.z - cst[2]), dy = (P.y - cst[1]) + (P.w - cst[3]);
        const float f1 = (float)v[2 * a] * sc, f2 = (float)v[2 * a + 1] * sc;
        ff_add_prod(h0, l0, sc, (float)v[2 * a]);
        ff_add_prod(h1, l1, sc, (float)v[2 * a + 1]);
        ff_add_prod(h2, l2, -dy, f1);
        ff_add_prod(h2, l2, dx, f2);
      }
    }
    block_sum_ff<B>(h0, l0, sh, &mom[0]);
    if (KIND == 1) {
      block_sum_ff<B>(h1, l1, sh, &mom[1]);
      block_sum_ff<B>(h2, l2, sh, &mom[2]);
    }
    if (threadIdx.x == 0 && alpha > 0.0) {  // completion weighted per body
      const double cf = alpha / g.len[i];
      mom[0] *= cf;
      mom[1] *= cf;
      if (KIND == 1) mom[2] *= alpha / g.W[i];
    }
    __syncthreads();
  }
  const double m0 = mom[0], m1 = mom[1], m2 = mom[2];
  for (int a = a0 + threadIdx.x; a < a1; a += B) {
    const double os = scaled ? g.sw[a] : 1.0;
    const double wk = g.w[a] * g.kappa[a];
    if (KIND == 0) {
      double k;
      if (pff) {
        const float2* __restrict__ pf2 = reinterpret_cast<const float2*>(partial);
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
        int s = 0;
        for (; s + 2 <= S; s += 2) {
          const float2 u = pf2[(long long)s * M + a], w2 = pf2[(long long)(s + 1) * M + a];
          ffadd(h0, l0, u.x, u.y);
          ffadd(h1, l1, w2.x, w2.y);
        }
        if (s < S) {
          const float2 u = pf2[(long long)s * M + a];
          ffadd(h0, l0, u.x, u.y);
        }
        ffadd(h0, l0, h1, l1);
        k = (double)h0 + (double)l0;
      } else {
        k = 0.0;
        for (int s = 0; s < S; ++s) k += partial[(long long)s * M + a];
      }
      out[a] = sign * (0.5 * v[a] + os * (m0 - kInv2Pi * k) - kInv4Pi * wk * v[a]);
    } else {
      double k1 = 0.0, k2 = 0.0;
      if (pff) {
        const float4* __restrict__ pf4 = reinterpret_cast<const float4*>(partial);
        float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
        for (int s = 0; s < S; ++s) {
          const float4 u = pf4[(long long)s * M + a];
          ffadd(h1, l1, u.x, u.y);
          ffadd(h2, l2, u.z, u.w);
        }
        k1 = (double)h1 + (double)l1;
        k2 = (double)h2 + (double)l2;
      } else {
        for (int s = 0; s < S; ++s) {
          const double2 p0 = reinterpret_cast<const double2*>(partial)[(long long)s * M + a];
          k1 += p0.x;
          k2 += p0.y;
        }
      }
      const double tx = -g.ny[a], ty = g.nx[a];
      const double v1 = v[2 * a], v2 = v[2 * a + 1];
      const double odd = -0.5 * kInvPi * wk * (tx * v1 + ty * v2);
      const double px = -(g.y[a] - yc), py = g.x[a] - xc;
      out[2 * a] = sign * (0.5 * v1 + os * (m0 + px * m2 - kInvPi * k1) + odd * tx);
      out[2 * a + 1] = sign * (0.5 * v2 + os * (m1 + py * m2 - kInvPi * k2) + odd * ty);
    }
  }
}

// Sum of the float-float partial slots of the FP32 pair sums, wide: a CTA
// takes 32 target entries x 8 slot groups; each thread adds slots g, g + 8, ...
// in float-float, the 8 group sums are combined in a fixed order
// (deterministic), and the total overwrites slot 0 as a double (the entry's
// own 8 bytes, after every thread has read it).  cw = float-float pairs per
// target entry (1 Laplace, 2 Stokes).
constexpr int kRT = 32, kRG = 8;

__global__ void __launch_bounds__(kRT * kRG) k_reduce_slots(double* __restrict__ partial, int S, long long n,
                                                            const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float sh[kRG][kRT], sl[kRG][kRT];
  const int tx = threadIdx.x % kRT, grp = threadIdx.x / kRT;
  const long long e = (long long)blockIdx.x * kRT + tx;  // a float-float entry
  const float2* __restrict__ pf2 = reinterpret_cast<const float2*>(partial);
  float h = 0.f, l = 0.f, h2 = 0.f, l2 = 0.f;
  if (e < n) {
    int s = grp;
    for (; s + kRG < S; s += 2 * kRG) {
      const float2 u = pf2[(long long)s * n + e], v = pf2[(long long)(s + kRG) * n + e];
      ffadd(h, l, u.x, u.y);
      ffadd(h2, l2, v.x, v.y);
    }
    if (s < S) {
      const float2 u = pf2[(long long)s * n + e];
      ffadd(h, l, u.x, u.y);
    }
    ffadd(h, l, h2, l2);
  }
  sh[grp][tx] = h;
  sl[grp][tx] = l;
  __syncthreads();
  if (grp == 0 && e < n) {
    float th = sh[0][tx], tl = sl[0][tx];
#pragma unroll
    for (int q = 1; q < kRG; ++q) ffadd(th, tl, sh[q][tx], sl[q][tx]);
    partial[e] = (double)th + (double)tl;
  }
}

// The same for FP64 partial slots (FP64 and float-float pair sums).
__global__ void __launch_bounds__(kRT * kRG) k_reduce_slots64(double* __restrict__ partial, int S, long long n,
                                                              const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ double sd[kRG][kRT];
  const int tx = threadIdx.x % kRT, grp = threadIdx.x / kRT;
  const long long e = (long long)blockIdx.x * kRT + tx;
  double a = 0.0, b = 0.0;
  if (e < n) {
    int s = grp;
    for (; s + kRG < S; s += 2 * kRG) {
      a += partial[(long long)s * n + e];
      b += partial[(long long)(s + kRG) * n + e];
    }
    if (s < S) a += partial[(long long)s * n + e];
  }
  sd[grp][tx] = a + b;
  __syncthreads();
  if (grp == 0 && e < n) {
    double t = sd[0][tx];
#pragma unroll
    for (int q = 1; q < kRG; ++q) t += sd[q][tx];
    partial[e] = t;
  }
}

// Right-hand side for a correction solved with the per-body weighted
// completion (weights c_i): for A e = g, the discrete Gauss identities (column
// sums of K equal -1/2 on the own body and 0 elsewhere, Sections 3.2 and 4.1)
// give the completion moments of e from g alone, L e = L~(g) with
// L~(g)_i = int_{Gamma_i} g / |Gamma_i| (and the torque moment over W_i), so
// A_c e = g - (I - C) L~(g).  Scaled vectors; one block per body.
template <int KIND>
__global__ void __launch_bounds__(kBE) k_consistent_rhs(Geo g, double alpha, const double* __restrict__ in,
                                                        double* __restrict__ out) {
  __shared__ double sh[kBE / 32];
  const int i = blockIdx.x;
  const int a0 = g.body_start[i], a1 = g.body_start[i + 1];
  const double xc = g.xc[i], yc = g.yc[i];
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for (int a = a0 + threadIdx.x; a < a1; a += kBE) {
    const double s = g.sw[a];
    if (KIND == 0) {
      m0 += s * in[a];
    } else {
      const double f1 = s * in[2 * a], f2 = s * in[2 * a + 1];
      m0 += f1;
      m1 += f2;
      m2 += -(g.y[a] - yc) * f1 + (g.x[a] - xc) * f2;
    }
  }
  m0 = block_sum<kBE>(m0, sh);
  if (KIND == 1) {
    m1 = block_sum<kBE>(m1, sh);
    m2 = block_sum<kBE>(m2, sh);
  }
  const double df = (1.0 - alpha / g.len[i]) / g.len[i];
  const double dt = KIND == 1 ? (1.0 - alpha / g.W[i]) / g.W[i] : 0.0;
  for (int a = a0 + threadIdx.x; a < a1; a += kBE) {
    const double s = g.sw[a];
    if (KIND == 0) {
      out[a] = in[a] - s * df * m0;
    } else {
      const double px = -(g.y[a] - yc), py = g.x[a] - xc;
      out[2 * a] = in[2 * a] - s * (df * m0 + dt * m2 * px);
      out[2 * a + 1] = in[2 * a + 1] - s * (df * m1 + dt * m2 * py);
    }
  }
}

// Occupancy of each pair kernel (blocks per SM) and the SM count, queried once
// per device.
struct DeviceShape {
  int nsm = 0;
  int occ[3][2] = {{0, 0}, {0, 0}, {0, 0}};  // [precision][kind]
};

// Per device, filled once under a lock: concurrent server threads must never
// see a half-filled entry (a different split count changes the summation
// order of the results).
const DeviceShape& device_shape() {
  static DeviceShape shapes[64];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  DeviceShape& d = shapes[dev & 63];
  std::lock_guard<std::mutex> lk(mu);
  if (d.nsm == 0) {
    DeviceShape t;
    cudaDeviceGetAttribute(&t.nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[0][0], k_pair64<0, false>, kB64, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[0][1], k_pair64<1, false>, kB64, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[1][0], k_pair32<0, false>, kB32, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[1][1], k_pair32<1, false>, kB32, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[2][0], k_pair_ff<0, false>, kBF, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t.occ[2][1], k_pair_ff<1, false>, kBF, 0);
    cudaGetLastError();
    if (t.nsm <= 0) t.nsm = 1;  // a failed query plans for one SM: slower, still correct
    for (auto& row : t.occ)
      for (int& o : row)
        if (o <= 0) o = 4;
    d = t;
  }
  return d;
}

}  // namespace

int device_sms() { return device_shape().nsm; }

// Choose the source split so that one wave fills every SM with as many
// blocks as can be resident: blocks = target blocks x splits ~ SMs x occupancy.
// Splits need not be tile-aligned (the kernels handle a short last tile).
namespace {

// Split counts chosen by timing (bie_tune), per device and shape (M, kind,
// precision); plan_pairs takes them before the occupancy rule.
std::mutex g_tune_mu;
std::map<std::array<int, 4>, PairPlan> g_tuned;

std::array<int, 4> tune_key(int M, int kind, int precision) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, M, kind, precision};
}

}  // namespace

void set_tuned_plan(int M, int kind, int precision, const PairPlan& p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[tune_key(M, kind, precision)] = p;
}

void forget_tuned_plan(int M, int kind, int precision) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.erase(tune_key(M, kind, precision));
}

void clear_tuned_splits() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
}

PairPlan plan_with_splits(int M, int S) {
  const long long cap = std::max(1, (M + 63) / 64);  // chunks of at least 64 sources
  long long s = std::min<long long>(std::max(S, 1), cap);
  const long long chunk = (M + s - 1) / s;
  return uniform_plan((int)((M + chunk - 1) / chunk), (int)chunk);
}

PairPlan plan_two_level(int M, int c1, int c2, double f) {
  c1 = std::max(64, c1);
  c2 = std::max(64, std::min(c1, c2));
  const int S1 = std::max(0, std::min((int)(f * M / c1), M / c1));
  const int rem = M - S1 * c1;
  if (rem <= 0) return uniform_plan(S1, c1);
  return PairPlan{S1 + (rem + c2 - 1) / c2, c1, S1, c2};
}

PairPlan plan_symmetric(int M) {
  PairPlan p = uniform_plan((M + kTS - 1) / kTS, kTS);
  p.sym = 1;
  return p;
}

PairPlan plan_pairs(int M, int kind, int precision) {
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(M, kind, precision));
    if (it != g_tuned.end()) return it->second;
  }
  return occupancy_plan(M, kind, precision);
}

PairPlan occupancy_plan(int M, int kind, int precision) {
  const DeviceShape& d = device_shape();
  if ((precision == 1 || precision == 2) && kind == 0) {
    // the symmetric FP32 / float-float Laplace kernels once their tile pairs fill
    // the GPU a few times over and their partials (one slot per tile) stay
    // within 256 MB
    const long long nt = (M + kTS - 1) / kTS;
    if (nt * (nt + 1) / 2 >= 4LL * d.nsm && nt * (long long)M * 8 <= (256LL << 20)) return plan_symmetric(M);
  }
  const int per_block = precision == 0 ? kB64 * kT64 : (precision == 1 ? kB32 * kT32 : kBF * kTF);
  const long long bx = (M + per_block - 1) / per_block;
  const long long slots = (long long)d.nsm * d.occ[precision][kind];
  long long S = bx >= slots ? 1 : slots / bx;
  const long long min_chunk = 64;
  if (S > (M + min_chunk - 1) / min_chunk) S = (M + min_chunk - 1) / min_chunk;
  if (S < 1) S = 1;
  const long long chunk = (M + S - 1) / S;
  return uniform_plan((int)((M + chunk - 1) / chunk), (int)chunk);
}

// Batched solves: target block x sums over the len_x nodes of its problems.
// With S splits of chunk = ceil(src_max / S) sources, block x has
// ceil(len_x / chunk) busy splits, each with about the same work whatever the
// problem's size.  S is the smallest count whose busy blocks fill every
// resident slot once (chunks of at least 64 sources).
PairPlan plan_pairs_batch(const int* body_start, int N, const int* pbody, int P, int kind, int precision) {
  const DeviceShape& d = device_shape();
  const int per_block = precision == 0 ? kB64 * kT64 : (precision == 1 ? kB32 * kT32 : kBF * kTF);
  const int M = body_start[N];
  std::vector<int> pstart(P + 1);
  int src_max = 1;
  for (int p = 0; p <= P; ++p) pstart[p] = p < P ? body_start[pbody[p]] : M;
  for (int p = 0; p < P; ++p) src_max = std::max(src_max, pstart[p + 1] - pstart[p]);
  const int bx = (M + per_block - 1) / per_block;
  std::vector<int> len(bx);
  for (int x = 0; x < bx; ++x) {
    const int tb = x * per_block, te = std::min(M, tb + per_block);
    const int p0 = (int)(std::upper_bound(pstart.begin(), pstart.end(), tb) - pstart.begin()) - 1;
    const int p1 = (int)(std::upper_bound(pstart.begin(), pstart.end(), te - 1) - pstart.begin()) - 1;
    len[x] = pstart[p1 + 1] - pstart[p0];
  }
  const long long slots = (long long)d.nsm * d.occ[precision][kind];
  const int s_cap = std::max(1, (src_max + 63) / 64);
  int S = 1;
  for (; S < s_cap; ++S) {
    const long long chunk = ((long long)src_max + S - 1) / S;
    long long busy = 0;
    for (int x = 0; x < bx; ++x) {
      const long long ch = std::max(chunk, ((long long)len[x] + S - 1) / S);
      busy += (len[x] + ch - 1) / ch;
    }
    if (busy >= slots) break;
  }
  return uniform_plan(S, (src_max + S - 1) / S);
}

namespace {

template <bool BATCH>
void launch_pairs(const Geo& g, int kind, int precision, const PairPlan& p, VecRef v, const double* sscale,
                  double* partial, const int* stop, cudaStream_t s) {
  if (precision == 0) {
    dim3 grid((g.M + kB64 * kT64 - 1) / (kB64 * kT64), p.S);
    if (kind == 0)
      k_pair64<0, BATCH><<<grid, kB64, 0, s>>>(g, v, sscale, p, partial, stop);
    else
      k_pair64<1, BATCH><<<grid, kB64, 0, s>>>(g, v, sscale, p, partial, stop);
  } else if (precision == 1) {
    dim3 grid((g.M + kB32 * kT32 - 1) / (kB32 * kT32), p.S);
    const int gs = (int)std::min<long long>(1216, (g.M + 255) / 256);
    if (kind == 0) {
      k_src32<0><<<gs, 256, 0, s>>>(g, v, sscale, stop);
      if (!BATCH && p.sym) {
        const long long nt = (g.M + kTS - 1) / kTS;
        k_pair32s<<<(unsigned)(nt * (nt + 1) / 2), kB32, 0, s>>>(g, (int)nt, partial, stop);
      } else {
        k_pair32<0, BATCH><<<grid, kB32, 0, s>>>(g, v, sscale, p, partial, stop);
      }
    } else {
      k_src32<1><<<gs, 256, 0, s>>>(g, v, sscale, stop);
      k_pair32<1, BATCH><<<grid, kB32, 0, s>>>(g, v, sscale, p, partial, stop);
    }
    note_launches(1);
  } else {
    dim3 grid((g.M + kBF * kTF - 1) / (kBF * kTF), p.S);
    if (kind == 0 && !BATCH && p.sym) {
      const long long nt = (g.M + kTileF - 1) / kTileF;
      k_pair_ffs<<<(unsigned)(nt * (nt + 1) / 2), kBFS, 0, s>>>(g, (int)nt, partial, sscale, v, stop);
    } else if (kind == 0)
      k_pair_ff<0, BATCH><<<grid, kBF, 0, s>>>(g, v, sscale, p, partial, stop);
    else
      k_pair_ff<1, BATCH><<<grid, kBF, 0, s>>>(g, v, sscale, p, partial, stop);
  }
}

}  // namespace

// Batched solves (g.prange set) run instances with the problem masks; a single
// problem runs instances without any of that code.
cudaError_t pair_sum(const Geo& g, int kind, int precision, const PairPlan& p, VecRef v,
                     const double* sscale, double* partial, const int* stop, cudaStream_t s) {
  if (g.prange)
    launch_pairs<true>(g, kind, precision, p, v, sscale, partial, stop, s);
  else
    launch_pairs<false>(g, kind, precision, p, v, sscale, partial, stop, s);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t epilogue(const Geo& g, int kind, const PairPlan& p, VecRef v, const double* partial,
                     int scaled, int with_L, double sign, VecRef out, const int* stop,
                     cudaStream_t s, double alpha, bool pff, bool fp32) {
  if (p.S >= kRG) {
    // add the slots wide first (float-float or FP64), then an epilogue over one FP64 slot
    const long long n = (long long)g.M * (kind + 1);
    const unsigned nb = (unsigned)((n + kRT - 1) / kRT);
    if (pff)
      k_reduce_slots<<<nb, kRT * kRG, 0, s>>>(const_cast<double*>(partial), p.S, n, stop);
    else
      k_reduce_slots64<<<nb, kRT * kRG, 0, s>>>(const_cast<double*>(partial), p.S, n, stop);
    note_launches(1);
    return epilogue(g, kind, uniform_plan(1, g.M), v, partial, scaled, with_L, sign, out, stop, s, alpha, false,
                    fp32);
  }
  // one block per body, sized to the bodies (many small bodies: small blocks)
  const int avg = g.M / std::max(1, g.N);
  const int pf = pff ? 1 : 0;
  if (fp32) {  // the FP32 operator: the epilogue in FP32 arithmetic
    if (avg <= 64) {
      if (kind == 0)
        k_epilogue32<0, 64><<<g.N, 64, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pf);
      else
        k_epilogue32<1, 64><<<g.N, 64, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pf);
    } else {
      if (kind == 0)
        k_epilogue32<0, kBE><<<g.N, kBE, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pf);
      else
        k_epilogue32<1, kBE><<<g.N, kBE, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pf);
    }
    note_launches(1);
    return cudaGetLastError();
  }
  if (avg <= 64) {
    if (kind == 0)
      k_epilogue<0, 64><<<g.N, 64, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pff ? 1 : 0);
    else
      k_epilogue<1, 64><<<g.N, 64, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pff ? 1 : 0);
  } else {
    if (kind == 0)
      k_epilogue<0, kBE><<<g.N, kBE, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pff ? 1 : 0);
    else
      k_epilogue<1, kBE><<<g.N, kBE, 0, s>>>(g, v, partial, p.S, scaled, with_L, alpha, sign, out, stop, pff ? 1 : 0);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t consistent_rhs(const Geo& g, int kind, double alpha, const double* in, double* out,
                           cudaStream_t s) {
  if (kind == 0)
    k_consistent_rhs<0><<<g.N, kBE, 0, s>>>(g, alpha, in, out);
  else
    k_consistent_rhs<1><<<g.N, kBE, 0, s>>>(g, alpha, in, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bie
