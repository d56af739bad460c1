// apply_operator_noalloc: the operator application of apply_operator for
// callers that cannot allocate device memory.
//
// Some callers must not allocate: code that runs under a memory budget fixed
// in advance, inside a framework that owns every device allocation through
// its own pool, or in a latency-critical loop where cudaMalloc/cudaFree (which
// may synchronise the device) are not allowed.  This entry point takes no
// context and allocates nothing: its scratch (the staged geometry and the
// pair-sum partials) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/bie2d.h"
#include "bie_internal.cuh"

using namespace bie;

namespace {

constexpr int kNoallocMaxNodes = BIE_NOALLOC_MAX_NODES;
constexpr int kNoallocMaxBodies = BIE_NOALLOC_MAX_BODIES;
constexpr int kNoallocMaxSplits = 16;
constexpr int kMaxDevices = 64;

// Bytes for: staged geometry (per node 7 doubles + 3 float4 + 3 float2 + 2 floats + int, per
// body 8 doubles + float4 + body_start) and the partials [splits][2 * nodes] doubles,
// each section padded to 256 bytes.
constexpr size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kScratchBytes =
    pad256((kNoallocMaxBodies + 1) * sizeof(int)) + pad256(kNoallocMaxNodes * sizeof(int)) +
    7 * pad256(kNoallocMaxNodes * sizeof(double)) + 3 * pad256(kNoallocMaxNodes * sizeof(float4)) +
    3 * pad256(kNoallocMaxNodes * sizeof(float2)) + pad256(2 * kNoallocMaxNodes * sizeof(float)) +
    8 * pad256(kNoallocMaxBodies * sizeof(double)) +
    pad256(kNoallocMaxBodies * sizeof(float4)) + pad256(2 * sizeof(double)) +
    pad256((size_t)kNoallocMaxSplits * 2 * kNoallocMaxNodes * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current (the host-side name of the array is only a stand-in).
std::mutex g_mu;
char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device memory of device `dev`, or managed memory.  Device memory of another
// GPU is refused: a kernel here would read it as a peer address (an illegal
// address without peer access).
bool device_ptr(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = pad256(off);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace

extern "C" int apply_operator_noalloc(const bie_geometry* geom, int kind, int precision, const double* in,
                                      double* out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!geom || !in || !out || !geom->body_start || !geom->x || !geom->y || !geom->dx || !geom->dy ||
      !geom->ddx || !geom->ddy)
    return BIE_ERR_INVALID;
  if (kind != BIE_KIND_LAPLACE && kind != BIE_KIND_STOKES) return BIE_ERR_INVALID;
  if (precision != BIE_PREC_FP64 && precision != BIE_PREC_MIXED && precision != BIE_PREC_MIXED_FF)
    return BIE_ERR_INVALID;
  const int N = geom->n_bodies;
  if (N < 1) return BIE_ERR_INVALID;
  if (N > kNoallocMaxBodies) return BIE_ERR_NOMEM;
  // every array must already be on the current device: nothing is staged
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return BIE_ERR_CUDA;
  }
  const void* arrays[] = {geom->body_start, geom->x, geom->y, geom->dx, geom->dy, geom->ddx, geom->ddy, in, out};
  for (const void* p : arrays)
    if (!device_ptr(p, cur)) return BIE_ERR_INVALID;
  if (geom->interior_pt && !device_ptr(geom->interior_pt, cur)) return BIE_ERR_INVALID;
  int bs_host[kNoallocMaxBodies + 1];
  if (cudaMemcpyAsync(bs_host, geom->body_start, (N + 1) * sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return BIE_ERR_CUDA;
  if (bs_host[0] != 0) return BIE_ERR_INVALID;
  for (int i = 0; i < N; ++i)
    if (bs_host[i + 1] - bs_host[i] < 8) return BIE_ERR_INVALID;
  const int M = bs_host[N];
  if (M > kNoallocMaxNodes) return BIE_ERR_NOMEM;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BIE_ERR_CUDA;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
        cudaGetLastError();
        return BIE_ERR_CUDA;
      }
      g_scratch_ptr[dev] = static_cast<char*>(p);
    }
    base = g_scratch_ptr[dev];
  }

  // carve the scratch exactly as the sizing above; every carved array is fully
  // written before it is read, so no section needs clearing
  Carver c{base};
  Geo g;
  g.N = N;
  g.M = M;
  int* body_start = c.take<int>(kNoallocMaxBodies + 1);
  g.body_of = c.take<int>(kNoallocMaxNodes);
  g.x = c.take<double>(kNoallocMaxNodes);
  g.y = c.take<double>(kNoallocMaxNodes);
  g.nx = c.take<double>(kNoallocMaxNodes);
  g.ny = c.take<double>(kNoallocMaxNodes);
  g.w = c.take<double>(kNoallocMaxNodes);
  g.sw = c.take<double>(kNoallocMaxNodes);
  g.kappa = c.take<double>(kNoallocMaxNodes);
  g.pf = c.take<float4>(kNoallocMaxNodes);
  g.nf = c.take<float2>(kNoallocMaxNodes);
  g.wkf = c.take<float2>(kNoallocMaxNodes);
  g.xff = c.take<float4>(kNoallocMaxNodes);
  g.xfl = c.take<float2>(kNoallocMaxNodes);
  g.nff = c.take<float4>(kNoallocMaxNodes);
  g.qf = c.take<float>(2 * kNoallocMaxNodes);
  g.len = c.take<double>(kNoallocMaxBodies);
  g.xc = c.take<double>(kNoallocMaxBodies);
  g.yc = c.take<double>(kNoallocMaxBodies);
  g.W = c.take<double>(kNoallocMaxBodies);
  g.zx = c.take<double>(kNoallocMaxBodies);
  g.zy = c.take<double>(kNoallocMaxBodies);
  g.delta = c.take<double>(kNoallocMaxBodies);
  g.wind = c.take<double>(kNoallocMaxBodies);
  g.bbox = c.take<float4>(kNoallocMaxBodies);
  g.qscale = c.take<double>(2);
  double* partial = c.take<double>((size_t)kNoallocMaxSplits * 2 * kNoallocMaxNodes);
  if (c.off > kScratchBytes) return BIE_ERR_NOMEM;  // sizing and carving disagree

  // the same source split as apply_operator, capped at the scratch's splits
  PairPlan p = plan_pairs(M, kind, precision);
  if (p.S > kNoallocMaxSplits) {
    const int tile = 256;
    int chunk = (M + kNoallocMaxSplits - 1) / kNoallocMaxSplits;
    chunk = (chunk + tile - 1) / tile * tile;
    p = uniform_plan((M + chunk - 1) / chunk, chunk);
  }
  if (cudaMemcpyAsync(body_start, geom->body_start, (N + 1) * sizeof(int), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return BIE_ERR_CUDA;
  g.body_start = body_start;
  if (stage_geometry(g, geom->x, geom->y, geom->dx, geom->dy, geom->ddx, geom->ddy, geom->interior_pt, s) !=
      cudaSuccess)
    return BIE_ERR_CUDA;
  VecRef vin = vec(const_cast<double*>(in));
  if (pair_sum(g, kind, precision, p, vin, g.w, partial, nullptr, s) != cudaSuccess) return BIE_ERR_CUDA;
  if (epilogue(g, kind, p, vin, partial, 0, 1, 1.0, vec(out), nullptr, s, 0.0, precision == BIE_PREC_MIXED) !=
      cudaSuccess)
    return BIE_ERR_CUDA;
  return BIE_OK;
}
