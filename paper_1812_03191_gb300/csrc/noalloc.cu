// noalloc.cu -- the force reduction of one level without any device allocation.
//
// Some callers cannot call cudaMalloc: a host whose device memory is entirely
// reserved by another allocator (a framework's caching allocator holding the whole
// budget), a latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation, or a sandboxed plug-in that is not allowed to allocate.  For
// them, df_force_level_noalloc computes the same per-level force as the context's
// force reduction, with its scratch (the per-block partial sums) in a fixed
// file-scope device array instead of memory the context allocates.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/dfnest.h"
#include "internal.h"

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxPartials = DF_NOALLOC_MAX_CELLS / kNaBlock;

// Scratch of every call on this device: 3 partial sums per block.  Static storage,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) double g_na_partials[3 * kNaMaxPartials];

// Device address of the array, looked up once per device (host code may not use
// the symbol's name as a device pointer).
std::mutex g_na_mu;
double* g_na_addr[64] = {};

__global__ void __launch_bounds__(kNaBlock)
    k_force_level_na(const double* __restrict__ rho, int n0, int n1, int n2, int G, int s0,
                     int s1, double lo0, double lo1, double lo2, double dx0, double dx1,
                     double dx2, int has_child, int co0, int co1, int co2, int ch0, int ch1,
                     int ch2, double GM, double eps, double rho0, int mirror, double mult,
                     double* partials) {
  __shared__ double sx[kNaBlock], sy[kNaBlock], sz[kNaBlock];
  long long t = blockIdx.x * (long long)kNaBlock + threadIdx.x;
  long long na = (long long)n0 * n1 * n2;
  double fx = 0.0, fy = 0.0, fz = 0.0;
  if (t < na) {
    int ai = (int)(t % n0), aj = (int)((t / n0) % n1), ak = (int)(t / ((long long)n0 * n1));
    bool covered = has_child && ai >= co0 && ai < co0 + ch0 && aj >= co1 && aj < co1 + ch1 &&
                   ak >= co2 && ak < co2 + ch2;
    if (!covered) {
      long long c = ((long long)(G + ak) * s1 + G + aj) * s0 + G + ai;
      double x = lo0 + (ai + 0.5) * dx0, y = lo1 + (aj + 0.5) * dx1, z = lo2 + (ak + 0.5) * dx2;
      double r2 = x * x + y * y + z * z + eps * eps;
      double inv3 = 1.0 / (r2 * sqrt(r2));
      double m = (rho[c] - rho0) * (dx0 * dx1 * dx2);
      // the unfolded domain across mirror planes: no component along a mirror axis,
      // mult copies of the simulated part for the others
      fx = mirror & 1 ? 0.0 : mult * (GM * m * x * inv3);
      fy = mirror & 2 ? 0.0 : mult * (GM * m * y * inv3);
      fz = mirror & 4 ? 0.0 : mult * (GM * m * z * inv3);
    }
  }
  sx[threadIdx.x] = fx;
  sy[threadIdx.x] = fy;
  sz[threadIdx.x] = fz;
  __syncthreads();
  for (int w = kNaBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sx[threadIdx.x] += sx[threadIdx.x + w];
      sy[threadIdx.x] += sy[threadIdx.x + w];
      sz[threadIdx.x] += sz[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x + 0] = sx[0];
    partials[3 * blockIdx.x + 1] = sy[0];
    partials[3 * blockIdx.x + 2] = sz[0];
  }
}

// fixed-order compensated (Neumaier) sum of the partials, one warp per component
__global__ void k_force_sum_na(const double* __restrict__ partials, int n, double* F_out) {
  int comp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s = 0.0, cmp = 0.0;
  for (int p = lane; p < n; p += 32) {
    double v = partials[3 * p + comp];
    double tt = s + v;
    cmp += fabs(s) >= fabs(v) ? (s - tt) + v : (v - tt) + s;
    s = tt;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double so = __shfl_down_sync(0xffffffffu, s, o);
    double co = __shfl_down_sync(0xffffffffu, cmp, o);
    if (lane < o) {
      double tt = s + so;
      cmp += fabs(s) >= fabs(so) ? (s - tt) + so : (so - tt) + s;
      s = tt;
      cmp += co;
    }
  }
  if (lane == 0) F_out[comp] = s + cmp;
}

}  // namespace

extern "C" int df_force_level_noalloc(const double* rho, const int n[3], int G,
                                      const double lo[3], const double dx[3],
                                      const int child_off[3], const int child_n[3], double GM,
                                      double eps, double rho0, int mirror, double* F_out,
                                      void* stream) {
  if (!rho || !n || !lo || !dx || !F_out)
    return dfn::set_error(DF_EINVAL, "df_force_level_noalloc: null argument");
  if (G < 0 || n[0] < 1 || n[1] < 1 || n[2] < 1 || !(dx[0] > 0) || !(dx[1] > 0) ||
      !(dx[2] > 0))
    return dfn::set_error(DF_EINVAL, "df_force_level_noalloc: bad sizes");
  long long cells = (long long)n[0] * n[1] * n[2];
  if (cells > DF_NOALLOC_MAX_CELLS)
    return dfn::set_error(DF_EINVAL,
                          "df_force_level_noalloc: %lld active cells exceed the fixed scratch "
                          "capacity of %d cells",
                          cells, DF_NOALLOC_MAX_CELLS);
  if ((child_off == nullptr) != (child_n == nullptr))
    return dfn::set_error(DF_EINVAL, "df_force_level_noalloc: give both child_off and child_n");
  if (child_off)
    for (int d = 0; d < 3; ++d)
      if (child_off[d] < 0 || child_n[d] < 1 || child_off[d] > n[d] - child_n[d])
        return dfn::set_error(DF_EINVAL,
                              "df_force_level_noalloc: covered box [%d, %d) outside the %d "
                              "active cells of axis %d",
                              child_off[d], child_off[d] + child_n[d], n[d], d);
  if (mirror < 0 || mirror > 7)
    return dfn::set_error(DF_EINVAL, "df_force_level_noalloc: mirror mask %d not in 0..7",
                          mirror);
  double mult = 1.0;
  for (int d = 0; d < 3; ++d)
    if (mirror >> d & 1) mult *= 2.0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return dfn::set_error(DF_ECUDA, "df_force_level_noalloc: no current device");
  double* partials;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_partials);
      if (e != cudaSuccess)
        return dfn::set_error(DF_ECUDA, "df_force_level_noalloc: cudaGetSymbolAddress: %s",
                              cudaGetErrorString(e));
      g_na_addr[dev] = (double*)p;
    }
    partials = g_na_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = (int)((cells + kNaBlock - 1) / kNaBlock);
  int s0 = n[0] + 2 * G, s1 = n[1] + 2 * G;
  int hc = child_off != nullptr;
  k_force_level_na<<<blocks, kNaBlock, 0, st>>>(
      rho, n[0], n[1], n[2], G, s0, s1, lo[0], lo[1], lo[2], dx[0], dx[1], dx[2], hc,
      hc ? child_off[0] : 0, hc ? child_off[1] : 0, hc ? child_off[2] : 0, hc ? child_n[0] : 0,
      hc ? child_n[1] : 0, hc ? child_n[2] : 0, GM, eps, rho0, mirror, mult, partials);
  k_force_sum_na<<<1, 96, 0, st>>>(partials, blocks, F_out);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return dfn::set_error(DF_ECUDA, "df_force_level_noalloc: launch: %s", cudaGetErrorString(e));
  return DF_OK;
}
