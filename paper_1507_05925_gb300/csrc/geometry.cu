// Geometry staging (quadrature data), incident densities, right-hand sides and
// output evaluation at interior points.  All FP64: these are O(M) or O(N M)
// passes off the per-iteration hot loop.
#include <math.h>

#include "bie_internal.cuh"
#include "logtab.cuh"
#include "reduce.cuh"

namespace bie {

namespace {

constexpr int kB = 256;

// One block per body.  Trapezoidal rule on theta_k = 2 pi k / n_i:
// w = |x'| 2pi/n_i, tau = x'/|x'|, n = (tau_y, -tau_x) (outward for CCW),
// kappa = (x' y'' - y' x'')/|x'|^3; per body |Gamma_i| = sum w, the arc-length
// centroid (Section 4, definition of x^c_i) and W_i = sum w |x - x^c|^2 (eq. rho).
__global__ void __launch_bounds__(kB) k_stage(Geo g, const double* __restrict__ X,
                                              const double* __restrict__ Y,
                                              const double* __restrict__ DX,
                                              const double* __restrict__ DY,
                                              const double* __restrict__ DDX,
                                              const double* __restrict__ DDY,
                                              const double* __restrict__ ipt) {
  __shared__ double sh[kB / 32];
  const int i = blockIdx.x;
  const int a0 = g.body_start[i], a1 = g.body_start[i + 1];
  const double hstep = 2.0 * kPi / (double)(a1 - a0);
  double sl = 0.0, sx = 0.0, sy = 0.0;
  double bx0 = 1e300, by0 = 1e300, bx1 = -1e300, by1 = -1e300;
  for (int a = a0 + threadIdx.x; a < a1; a += kB) {
    const double x = X[a], y = Y[a], dx = DX[a], dy = DY[a];
    const double sp = sqrt(dx * dx + dy * dy);
    const double w = sp * hstep;
    const double tx = dx / sp, ty = dy / sp;
    const double kap = (dx * DDY[a] - dy * DDX[a]) / (sp * sp * sp);
    g.x[a] = x;
    g.y[a] = y;
    g.nx[a] = ty;
    g.ny[a] = -tx;
    g.w[a] = w;
    const double sw = sqrt(w);
    g.sw[a] = sw;
    g.kappa[a] = kap;
    const float xh = (float)x, yh = (float)y;
    g.pf[a] = make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
    g.nf[a] = make_float2((float)ty, (float)(-tx));
    g.wkf[a] = make_float2((float)sw, (float)(w * kap));
    g.body_of[a] = i;
    sl += w;
    sx += w * x;
    sy += w * y;
    bx0 = fmin(bx0, x);
    by0 = fmin(by0, y);
    bx1 = fmax(bx1, x);
    by1 = fmax(by1, y);
  }
  bx0 = block_min<kB>(bx0, sh);
  by0 = block_min<kB>(by0, sh);
  bx1 = -block_min<kB>(-bx1, sh);
  by1 = -block_min<kB>(-by1, sh);
  sl = block_sum<kB>(sl, sh);
  sx = block_sum<kB>(sx, sh);
  sy = block_sum<kB>(sy, sh);
  const double xc = sx / sl, yc = sy / sl;
  const double zx = ipt ? ipt[2 * i] : xc;
  const double zy = ipt ? ipt[2 * i + 1] : yc;
  double sW = 0.0, dmin2 = 1e300, wind = 0.0;
  for (int a = a0 + threadIdx.x; a < a1; a += kB) {
    const double ux = X[a] - xc, uy = Y[a] - yc;
    sW += g.w[a] * (ux * ux + uy * uy);
    const double px = X[a] - zx, py = Y[a] - zy;
    dmin2 = fmin(dmin2, px * px + py * py);
    const int b = (a + 1 < a1) ? a + 1 : a0;
    const double qx = X[b] - zx, qy = Y[b] - zy;
    wind += atan2(px * qy - py * qx, px * qx + py * qy);
  }
  sW = block_sum<kB>(sW, sh);
  wind = block_sum<kB>(wind, sh);
  dmin2 = block_min<kB>(dmin2, sh);
  if (threadIdx.x == 0) {
    g.len[i] = sl;
    g.xc[i] = xc;
    g.yc[i] = yc;
    g.W[i] = sW;
    g.zx[i] = zx;
    g.zy[i] = zy;
    g.delta[i] = 0.25 * sqrt(dmin2);
    g.wind[i] = wind / (2.0 * kPi);
    // rounded outwards to FP32
    g.bbox[i] = make_float4(__double2float_rd(bx0), __double2float_rd(by0), __double2float_ru(bx1),
                            __double2float_ru(by1));
  }
}

// Quanta for the exact three-float split of positions used by the
// float-float pair sums: with |x| < 2^e for every coordinate, Q = 22 - e, so
// x = h + m + l with h a multiple of 2^-Q (|h| 2^Q < 2^22), m a multiple of
// 2^-(Q+23) and |l| <= 2^-(Q+24): differences of h's and of m's are exact.
__global__ void k_geo_scale(Geo g) {
  __shared__ double sh[kB / 32];
  double m = 0.0;
  for (int i = threadIdx.x; i < g.N; i += kB) {
    const float4 b = g.bbox[i];
    m = fmax(m, fmax(fmax(fabs((double)b.x), fabs((double)b.y)), fmax(fabs((double)b.z), fabs((double)b.w))));
  }
  m = -block_min<kB>(-m, sh);
  if (threadIdx.x == 0) {
    int e = 0;
    frexp(fmax(m, 1e-300), &e);  // m < 2^e
    g.qscale[0] = ldexp(1.0, 22 - e);
    g.qscale[1] = ldexp(1.0, 45 - e);
  }
}

// Per-node splits for the float-float pair sums: positions x = h + m + l on
// the quanta of qscale (multiplying by the inverse quantum, a power of two,
// is exact), normals n = h + l.
__global__ void k_geo_split(Geo g) {
  const double s0 = g.qscale[0], s1 = g.qscale[1];
  const double i0 = 1.0 / s0, i1 = 1.0 / s1;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.M; a += gridDim.x * blockDim.x) {
    float h[2], m[2], l[2];
    const double c[2] = {g.x[a], g.y[a]};
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const double hh = rint(c[d] * s0) * i0;
      const double r = c[d] - hh;
      const double mm = rint(r * s1) * i1;
      h[d] = (float)hh;
      m[d] = (float)mm;
      l[d] = (float)(r - mm);
    }
    g.xff[a] = make_float4(h[0], m[0], h[1], m[1]);
    g.xfl[a] = make_float2(l[0], l[1]);
    const double nx = g.nx[a], ny = g.ny[a];
    const float nxh = (float)nx, nyh = (float)ny;
    g.nff[a] = make_float4(nxh, (float)(nx - (double)nxh), nyh, (float)(ny - (double)nyh));
  }
}

// f = sw * (L sigma): q_i on Gamma_i (Laplace), F_i + T_i (x - x^c_i)^perp (Stokes).
__global__ void k_total_rhs(Geo g, int kind, const double* __restrict__ load, double* __restrict__ f) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.M; a += gridDim.x * blockDim.x) {
    const int i = g.body_of[a];
    const double s = g.sw[a];
    if (kind == 0) {
      f[a] = s * load[i];
    } else {
      const double px = -(g.y[a] - g.yc[i]), py = g.x[a] - g.xc[i];
      const double F1 = load[3 * i], F2 = load[3 * i + 1], T = load[3 * i + 2];
      f[2 * a] = s * (F1 + T * px);
      f[2 * a + 1] = s * (F2 + T * py);
    }
  }
}

// sw * sigma, sigma_a = q_i/|Gamma_i| (eq. sigma); sw * rho,
// rho_a = F_i/|Gamma_i| + T_i (x_a - x^c_i)^perp / W_i (eq. rho).
__global__ void k_incident(Geo g, int kind, const double* __restrict__ load, double* __restrict__ out) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < g.M; a += gridDim.x * blockDim.x) {
    const int i = g.body_of[a];
    const double s = g.sw[a];
    if (kind == 0) {
      out[a] = s * (load[i] / g.len[i]);
    } else {
      const double px = -(g.y[a] - g.yc[i]), py = g.x[a] - g.xc[i];
      const double T = load[3 * i + 2];
      out[2 * a] = s * (load[3 * i] / g.len[i] + T * px / g.W[i]);
      out[2 * a + 1] = s * (load[3 * i + 1] / g.len[i] + T * py / g.W[i]);
    }
  }
}

__global__ void k_unscale(Geo g, int comps, const double* __restrict__ v, double* __restrict__ out) {
  const long long n = (long long)g.M * comps;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = v[k] / g.sw[k / comps];
}

__global__ void k_scale_by(int M, int comps, const double* __restrict__ in, const double* __restrict__ fac,
                           double* __restrict__ out) {
  const long long n = (long long)M * comps;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = in[k] * fac[k / comps];
}

// Net load |sum_i q_i| (or |sum_i F_i|) and max |load| over bodies [i0, i1)
// (block-wide; valid in every thread).
__device__ __forceinline__ double2 net_and_max(int kind, const double* __restrict__ load, int i0, int i1,
                                               double* sh) {
  double s0 = 0, s1 = 0, nmx = 0;  // nmx: -max |load|
  for (int i = i0 + threadIdx.x; i < i1; i += kB) {
    if (kind == 0) {
      s0 += load[i];
      nmx = fmin(nmx, -fabs(load[i]));
    } else {
      s0 += load[3 * i];
      s1 += load[3 * i + 1];
      nmx = fmin(nmx, -fmax(fabs(load[3 * i]), fmax(fabs(load[3 * i + 1]), fabs(load[3 * i + 2]))));
    }
  }
  s0 = block_sum<kB>(s0, sh);
  s1 = block_sum<kB>(s1, sh);
  nmx = block_min<kB>(nmx, sh);
  return make_double2(sqrt(s0 * s0 + s1 * s1), -nmx);
}

// One problem: out = (net load, max |load|).
__global__ void __launch_bounds__(kB) k_net_load(int N, int kind, const double* __restrict__ load,
                                                  double* __restrict__ out) {
  __shared__ double sh[kB / 32];
  const double2 r = net_and_max(kind, load, 0, N, sh);
  if (threadIdx.x == 0) {
    out[0] = r.x;
    out[1] = r.y;
  }
}

// Batched solves, one block per problem p (bodies pbody[p]..pbody[p+1]):
// per[2p] = its net load, per[2p+1] = its max |load|.
__global__ void __launch_bounds__(kB) k_net_load_batch(int kind, const double* __restrict__ load,
                                                        const int* __restrict__ pbody, double* __restrict__ per) {
  __shared__ double sh[kB / 32];
  const int p = blockIdx.x;
  const double2 r = net_and_max(kind, load, pbody[p], pbody[p + 1], sh);
  if (threadIdx.x == 0) {
    per[2 * p] = r.x;
    per[2 * p + 1] = r.y;
  }
}

// out = (largest net load, largest |load|) over the P problems.
__global__ void __launch_bounds__(kB) k_net_load_max(const double* __restrict__ per, int P, double* __restrict__ out) {
  __shared__ double sh[kB / 32];
  double a = 0.0, b = 0.0;
  for (int p = threadIdx.x; p < P; p += kB) {
    a = fmax(a, per[2 * p]);
    b = fmax(b, per[2 * p + 1]);
  }
  a = -block_min<kB>(-a, sh);
  b = -block_min<kB>(-b, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// Batched solves: scale each problem's entries [pnode[p], pnode[p+1]) of f to
// unit 2-norm (scale[p] = the norm, 1 for a zero segment), or multiply them
// back by scale[p].
__global__ void __launch_bounds__(kB) k_batch_normalize(double* __restrict__ f, const long long* __restrict__ pnode,
                                                        double* __restrict__ scale) {
  __shared__ double sh[kB / 32];
  const int p = blockIdx.x;
  const long long e0 = pnode[p], e1 = pnode[p + 1];
  double s = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += kB) s += f[e] * f[e];
  s = sqrt(block_sum<kB>(s, sh));
  const double sc = s > 0.0 ? s : 1.0;
  const double inv = 1.0 / sc;
  for (long long e = e0 + threadIdx.x; e < e1; e += kB) f[e] *= inv;
  if (threadIdx.x == 0) scale[p] = sc;
}

__global__ void __launch_bounds__(kB) k_batch_unscale(double* __restrict__ x, const long long* __restrict__ pnode,
                                                      const double* __restrict__ scale) {
  const int p = blockIdx.x;
  const double sc = scale[p];
  for (long long e = pnode[p] + threadIdx.x; e < pnode[p + 1]; e += kB) x[e] *= sc;
}

__global__ void __launch_bounds__(kB) k_gather(const CopySeg* __restrict__ segs, int nseg) {
  for (int i = blockIdx.x; i < nseg; i += gridDim.x) {
    const CopySeg sg = segs[i];
    const unsigned* __restrict__ src = static_cast<const unsigned*>(sg.src);
    unsigned* __restrict__ dst = static_cast<unsigned*>(sg.dst);
    for (long long k = threadIdx.x; k < sg.words; k += kB) dst[k] = src[k];
  }
}

// Batched solves: ||x_p|| of every problem's entries into norms[p].
__global__ void __launch_bounds__(kB) k_seg_norms(const double* __restrict__ x, const long long* __restrict__ pnode,
                                                  double* __restrict__ norms) {
  __shared__ double sh[kB / 32];
  const int p = blockIdx.x;
  double s = 0.0;
  for (long long e = pnode[p] + threadIdx.x; e < pnode[p + 1]; e += kB) s += x[e] * x[e];
  s = block_sum<kB>(s, sh);
  if (threadIdx.x == 0) norms[p] = sqrt(s);
}

// Batched solves: x_p = 0 for every problem with norms[p] <= thr.
__global__ void __launch_bounds__(kB) k_seg_zero_below(double* __restrict__ x, const long long* __restrict__ pnode,
                                                       const double* __restrict__ norms, double thr) {
  const int p = blockIdx.x;
  if (!(norms[p] <= thr)) return;
  for (long long e = pnode[p] + threadIdx.x; e < pnode[p + 1]; e += kB) x[e] = 0.0;
}

// Laplace single layer at z_i: sum_b w_b nu_b log|z_i - x_b|^2 over split p.
__global__ void __launch_bounds__(kB) k_out_lap(Geo g, const double* __restrict__ v,
                                                double* __restrict__ part, int P) {
  __shared__ double sh[kB / 32];
  __shared__ double2 ltab[kLogTab];
  log_table_fill(ltab);
  __syncthreads();
  const int i = blockIdx.x, p = blockIdx.y;
  const double zx = g.zx[i], zy = g.zy[i];
  // sources: all nodes, or the nodes of body i's problem (batched solves)
  const int s0 = g.prange ? g.prange[i].x : 0, s1 = g.prange ? g.prange[i].y : g.M;
  const int chunk = (s1 - s0 + P - 1) / P;
  const int b0 = s0 + p * chunk, b1 = min(s1, b0 + chunk);
  double acc = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += kB) {
    const double rx = zx - g.x[b], ry = zy - g.y[b];
    acc += g.sw[b] * v[b] * log_tab(rx * rx + ry * ry, ltab);
  }
  acc = block_sum<kB>(acc, sh);
  if (threadIdx.x == 0) part[(long long)p * g.N + i] = acc;
}

// Stokes single layer (Stokeslet G_ij = (1/4pi)[-log r d_ij + r_i r_j / r^2]) at
// the three stencil points of body i: t = 3i + s, s = 0: z0, 1: z0 + delta e1,
// 2: z0 + delta e2.
__global__ void __launch_bounds__(kB) k_out_stk(Geo g, const double* __restrict__ v,
                                                double* __restrict__ part, int P) {
  __shared__ double sh[kB / 32];
  __shared__ double2 ltab[kLogTab];
  log_table_fill(ltab);
  __syncthreads();
  const int t = blockIdx.x, p = blockIdx.y;
  const int i = t / 3, s = t % 3;
  const double d = g.delta[i];
  const double zx = g.zx[i] + (s == 1 ? d : 0.0), zy = g.zy[i] + (s == 2 ? d : 0.0);
  const int s0 = g.prange ? g.prange[i].x : 0, s1 = g.prange ? g.prange[i].y : g.M;
  const int chunk = (s1 - s0 + P - 1) / P;
  const int b0 = s0 + p * chunk, b1 = min(s1, b0 + chunk);
  double u1 = 0.0, u2 = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += kB) {
    const double rx = zx - g.x[b], ry = zy - g.y[b];
    const double r2 = rx * rx + ry * ry;
    const double f1 = g.sw[b] * v[2 * b], f2 = g.sw[b] * v[2 * b + 1];
    const double lg = -0.5 * log_tab(r2, ltab);
    const double c = (rx * f1 + ry * f2) / r2;
    u1 += lg * f1 + c * rx;
    u2 += lg * f2 + c * ry;
  }
  u1 = block_sum<kB>(u1, sh);
  u2 = block_sum<kB>(u2, sh);
  if (threadIdx.x == 0) {
    part[((long long)p * 3 * g.N + t) * 2] = u1;
    part[((long long)p * 3 * g.N + t) * 2 + 1] = u2;
  }
}

// One block per body: combine the splits, form the outputs, and measure the
// constraint residuals int_{Gamma_i} mu = int nu - q_i (Laplace) or the force
// and torque moments of mu = nu - rho (Stokes).
__global__ void __launch_bounds__(kB) k_out_final(Geo g, int kind, const double* __restrict__ v,
                                                  const double* __restrict__ load,
                                                  const double* __restrict__ part, int P,
                                                  double* __restrict__ out, double* __restrict__ cbody) {
  __shared__ double sh[kB / 32];
  const int i = blockIdx.x;
  const int a0 = g.body_start[i], a1 = g.body_start[i + 1];
  double m0 = 0.0, m1 = 0.0, m2 = 0.0;
  for (int a = a0 + threadIdx.x; a < a1; a += kB) {
    if (kind == 0) {
      m0 += g.sw[a] * v[a];
    } else {
      const double f1 = g.sw[a] * v[2 * a], f2 = g.sw[a] * v[2 * a + 1];
      const double px = -(g.y[a] - g.yc[i]), py = g.x[a] - g.xc[i];
      m0 += f1;
      m1 += f2;
      m2 += px * f1 + py * f2;
    }
  }
  m0 = block_sum<kB>(m0, sh);
  if (kind == 1) {
    m1 = block_sum<kB>(m1, sh);
    m2 = block_sum<kB>(m2, sh);
  }
  if (threadIdx.x == 0) {
    if (kind == 0) {
      double acc = 0.0;
      for (int p = 0; p < P; ++p) acc += part[(long long)p * g.N + i];
      out[i] = -0.5 * kInv2Pi * acc;
      cbody[i] = fabs(m0 - load[i]);
    } else {
      double u[3][2] = {{0, 0}, {0, 0}, {0, 0}};
      for (int p = 0; p < P; ++p)
        for (int s = 0; s < 3; ++s) {
          u[s][0] += part[((long long)p * 3 * g.N + 3 * i + s) * 2];
          u[s][1] += part[((long long)p * 3 * g.N + 3 * i + s) * 2 + 1];
        }
      for (int s = 0; s < 3; ++s) {
        u[s][0] *= kInv4Pi;
        u[s][1] *= kInv4Pi;
      }
      const double d = g.delta[i];
      out[3 * i] = u[0][0];
      out[3 * i + 1] = u[0][1];
      out[3 * i + 2] = ((u[1][1] - u[0][1]) - (u[2][0] - u[0][0])) / (2.0 * d);
      cbody[i] = fmax(fabs(m0 - load[3 * i]), fmax(fabs(m1 - load[3 * i + 1]), fabs(m2 - load[3 * i + 2])));
    }
  }
}

__global__ void k_max_reduce(const double* __restrict__ c, int N, const double* __restrict__ netload,
                             double* __restrict__ out) {
  __shared__ double sh[kB / 32];
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += kB) m = fmax(m, c[i]);
  m = -block_min<kB>(-m, sh);
  if (threadIdx.x == 0) out[0] = m / fmax(netload[1], 1e-300);
}

inline int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

cudaError_t stage_geometry(const Geo& g, const double* x, const double* y, const double* dx,
                           const double* dy, const double* ddx, const double* ddy,
                           const double* interior_pt, cudaStream_t s) {
  k_stage<<<g.N, kB, 0, s>>>(g, x, y, dx, dy, ddx, ddy, interior_pt);
  note_launches(1);
  k_geo_scale<<<1, kB, 0, s>>>(g);
  note_launches(1);
  k_geo_split<<<grid_for(g.M), 256, 0, s>>>(g);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t total_density_rhs(const Geo& g, int kind, const double* load, double* f, cudaStream_t s) {
  k_total_rhs<<<grid_for(g.M), 256, 0, s>>>(g, kind, load, f);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t incident_density_scaled(const Geo& g, int kind, const double* load, double* out,
                                    cudaStream_t s) {
  k_incident<<<grid_for(g.M), 256, 0, s>>>(g, kind, load, out);
  note_launches(1);
  return cudaGetLastError();
}

int output_splits(const Geo& g, int kind) {
  const int targets = kind == 0 ? g.N : 3 * g.N;
  int P = (4 * device_sms() + targets - 1) / targets;
  const int maxP = (g.M + 255) / 256;
  if (P > maxP) P = maxP;
  if (P < 1) P = 1;
  return P;
}

cudaError_t finalize_output(const Geo& g, int kind, const double* v, const double* load, double* partial, int P,
                            double* out, double* cres, cudaStream_t s) {
  const int targets = kind == 0 ? g.N : 3 * g.N;
  double* cbody = partial + (long long)P * targets * (kind == 0 ? 1 : 2);
  double* nl = cbody + g.N;
  k_out_final<<<g.N, kB, 0, s>>>(g, kind, v, load, partial, P, out, cbody);
  note_launches(1);
  if (g.pbody && g.pnet) {
    k_net_load_batch<<<g.nprob, kB, 0, s>>>(kind, load, g.pbody, g.pnet);
    k_net_load_max<<<1, kB, 0, s>>>(g.pnet, g.nprob, nl);
    note_launches(2);
  } else {
    k_net_load<<<1, kB, 0, s>>>(g.N, kind, load, nl);
    note_launches(1);
  }
  k_max_reduce<<<1, kB, 0, s>>>(cbody, g.N, nl, cres);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t evaluate_output(const Geo& g, int kind, const double* v, const double* load,
                            double* partial, int P, double* out, double* cres, cudaStream_t s) {
  // partial: [P][targets][comps] followed by N per-body constraint residuals and
  // two net-load scalars
  if (kind == 0)
    k_out_lap<<<dim3(g.N, P), kB, 0, s>>>(g, v, partial, P);
  else
    k_out_stk<<<dim3(3 * g.N, P), kB, 0, s>>>(g, v, partial, P);
  note_launches(1);
  return finalize_output(g, kind, v, load, partial, P, out, cres, s);
}

cudaError_t unscale(const Geo& g, int kind, const double* v, double* out, cudaStream_t s) {
  k_unscale<<<grid_for((long long)g.M * (kind + 1)), 256, 0, s>>>(g, kind + 1, v, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t scale_by(const Geo& g, int kind, const double* in, const double* fac, double* out,
                     cudaStream_t s) {
  k_scale_by<<<grid_for((long long)g.M * (kind + 1)), 256, 0, s>>>(g.M, kind + 1, in, fac, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t batch_normalize(int nprob, const long long* pnode, double* f, double* scale, cudaStream_t s) {
  k_batch_normalize<<<nprob, kB, 0, s>>>(f, pnode, scale);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t batch_unscale(int nprob, const long long* pnode, const double* scale, double* x, cudaStream_t s) {
  k_batch_unscale<<<nprob, kB, 0, s>>>(x, pnode, scale);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t gather_segments(const std::vector<CopySeg>& segs, cudaStream_t s) {
  if (segs.empty()) return cudaSuccess;
  CopySeg* d = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&d), segs.size() * sizeof(CopySeg), s);
  if (e != cudaSuccess) return e;
  // a pageable source: the call returns once the table is staged
  e = cudaMemcpyAsync(d, segs.data(), segs.size() * sizeof(CopySeg), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const int n = (int)segs.size();
    k_gather<<<n < 1024 ? n : 1024, kB, 0, s>>>(d, n);
    note_launches(1);
    e = cudaGetLastError();
  }
  const cudaError_t f = cudaFreeAsync(d, s);
  return e != cudaSuccess ? e : f;
}

cudaError_t seg_norms(int nprob, const long long* pnode, const double* x, double* norms, cudaStream_t s) {
  k_seg_norms<<<nprob, kB, 0, s>>>(x, pnode, norms);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t seg_zero_below(int nprob, const long long* pnode, const double* norms, double thr, double* x,
                           cudaStream_t s) {
  k_seg_zero_below<<<nprob, kB, 0, s>>>(x, pnode, norms, thr);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t net_load(int N, int kind, const double* load, double* out, cudaStream_t s) {
  k_net_load<<<1, kB, 0, s>>>(N, kind, load, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace bie

namespace bie {
namespace {
__global__ void __launch_bounds__(256) k_test_log(const double* __restrict__ x, long long n, double* __restrict__ out) {
  __shared__ double2 ltab[kLogTab];
  log_table_fill(ltab);
  __syncthreads();
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    out[i] = log_tab(x[i], ltab);
    out[n + i] = log(x[i]);
  }
}
}  // namespace
}  // namespace bie

extern "C" int bie_test_log(const double* x, double* out, long long n, void* stream) {
  if (!x || !out || n < 0) return BIE_ERR_INVALID;
  if (n == 0) return BIE_OK;
  const long long b = (n + 255) / 256;
  bie::k_test_log<<<(unsigned)(b > 4096 ? 4096 : b), 256, 0, (cudaStream_t)stream>>>(x, n, out);
  bie::note_launches(1);
  return cudaGetLastError() == cudaSuccess ? BIE_OK : BIE_ERR_CUDA;
}
