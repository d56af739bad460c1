// Per-pair arithmetic shared by the direct pair sums and the FMM near field.
//
// A pair contributes c(r) r to the target's accumulator, r = x_a - x_b:
//   Laplace  c = q_b / |r|^2                    (the target dots the sum with n_a)
//   Stokes   c = (r . q_b)(r . n_a) / |r|^4     (q_b = w_b mu_b, a 2-vector)
// The kernel constants, the diagonal and the completion are applied later.
#pragma once

#include <cuda_runtime.h>

namespace bie {

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ------------------------------------------------------------------- FP32 ----
// Contribution of one pair from hi/lo positions (x = hi + lo): the leading
// difference is exact, so r . n_a keeps its digits for neighbouring nodes.
template <int KIND>
__device__ __forceinline__ void f32_pair(float txh, float tyh, float txl, float tyl, float tnx, float tny,
                                         float4 p, float q1, float q2, float& cx, float& cy) {
  const float dx = (txh - p.x) + (txl - p.z);
  const float dy = (tyh - p.y) + (tyl - p.w);
  const float r2 = fmaf(dx, dx, dy * dy);
  const float inv = rcp_approx(r2);
  float c;
  if (KIND == 0) {
    c = q1 * inv;
  } else {
    const float rq = fmaf(dx, q1, dy * q2);
    const float rn = fmaf(dx, tnx, dy * tny);
    c = (rq * rn) * (inv * inv);
  }
  cx = c * dx;
  cy = c * dy;
}

// ------------------------------------------------------------ float-float ----
// Every quantity is an unevaluated sum h + l of two floats (about 48 bits).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (ah + al)(bh + bl) as an unevaluated pair (p, e), |e| <~ 2^-22 |p|
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& p, float& e) {
  p = ah * bh;
  e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, fmaf(al, bh, e));
}

// float-float difference of two exactly split coordinates (h, m on common quanta)
__device__ __forceinline__ void ff_diff(float ah, float am, float al, float bh, float bm, float bl, float& dh,
                                        float& dl) {
  const float d1 = ah - bh;  // exact: multiples of 2^-Q below 2^23 quanta
  const float d2 = am - bm;  // exact likewise
  dh = d1 + d2;              // |d1| >= |d2| unless d1 = 0: fast two-sum
  dl = (d2 - (dh - d1)) + (al - bl);
}

// (sh, sl) += (th, tl)
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float th, float tl) {
  float u, e;
  two_sum(sh, th, u, e);
  sh = u;
  sl += e + tl;
}

// Target data of the float-float pair: position split (h, m, l) per
// coordinate and the normal (h, l) per component.
struct FFTarget {
  float xh, xm, xl, yh, ym, yl;
  float4 n;  // (nx_h, nx_l, ny_h, ny_l)
};

// Contribution (cx, cy) of one pair in float-float: sa = (xh, xm, yh, ym),
// sb = (xl, yl), q = (q1h, q1l, q2h, q2l).  Products are error-free (FMA),
// 1/r2 is the MUFU reciprocal refined by one float-float Newton step.
template <int KIND>
__device__ __forceinline__ void ff_pair(const FFTarget& t, float4 sa, float2 sb, float4 q, float& cxh, float& cxl,
                                        float& cyh, float& cyl) {
  float dxh, dxl, dyh, dyl;
  ff_diff(t.xh, t.xm, t.xl, sa.x, sa.y, sb.x, dxh, dxl);
  ff_diff(t.yh, t.ym, t.yl, sa.z, sa.w, sb.y, dyh, dyl);
  // r2 = dx^2 + dy^2: error-free squares, Fast2Sum of the two (both >= 0,
  // ordered by max/min), then the cross terms and renormalisation
  const float p1 = dxh * dxh, p1e = fmaf(dxh, dxh, -p1);
  const float p2 = dyh * dyh, p2e = fmaf(dyh, dyh, -p2);
  const float s = p1 + p2;
  const float se = fminf(p1, p2) - (s - fmaxf(p1, p2));
  const float lo = fmaf(2.0f, fmaf(dxh, dxl, dyh * dyl), (se + p1e) + p2e);
  const float r2h = s + lo;
  const float r2l = lo - (r2h - s);
  const float y0 = rcp_approx(r2h);
  const float ee = fmaf(-r2l, y0, fmaf(-r2h, y0, 1.0f));
  const float il = y0 * ee;
  float ch, cl;
  if (KIND == 0) {
    ff_mul(q.x, q.y, y0, il, ch, cl);
  } else {
    float rqh, rql, rnh, rnl, t1, t1e, t2, t2e, i2h, i2l, uh, ul;
    ff_mul(dxh, dxl, q.x, q.y, t1, t1e);
    ff_mul(dyh, dyl, q.z, q.w, t2, t2e);
    two_sum(t1, t2, rqh, rql);
    rql += t1e + t2e;
    ff_mul(dxh, dxl, t.n.x, t.n.y, t1, t1e);
    ff_mul(dyh, dyl, t.n.z, t.n.w, t2, t2e);
    two_sum(t1, t2, rnh, rnl);
    rnl += t1e + t2e;
    ff_mul(y0, il, y0, il, i2h, i2l);
    ff_mul(rqh, rql, rnh, rnl, uh, ul);
    ff_mul(uh, ul, i2h, i2l, ch, cl);
  }
  ff_mul(ch, cl, dxh, dxl, cxh, cxl);
  ff_mul(ch, cl, dyh, dyl, cyh, cyl);
}

}  // namespace bie
