// dfnest.cu -- host runtime and C ABI of libdfnest.so (see include/dfnest.h).
//
// The hierarchy of Sec. 3 lives on one GPU: one padded allocation per field per
// level, one scratch set shared by all levels (they are advanced one at a time),
// device scalars for the time step, time, force and health flag.  One coarse step
// (Eq. 55 time step, the Sec. 3.3 recursion, the Eq. 18 force) is issued as a
// fixed launch sequence that is captured once into a CUDA graph and replayed; the
// time step is read by the kernels from device memory, so nothing syncs the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/dfnest.h"
#include "internal.h"

using namespace dfn;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(DF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

// reach of one level step in cells along any axis (measured by perturbation
// propagation on the same scheme: G = 2 * reach is the smallest exact ghost width)
constexpr int kReach = 4;

struct Level {
  LevelView v;
  void* mem = nullptr;
  double* acc = nullptr;
  size_t acc_elems = 0;
};

}  // namespace

int dfn::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

struct df_ctx {
  int nl = 0, prec = 0, device = 0, G = 0;
  int n[3] = {0, 0, 0};
  double lo[3], hi[3];
  size_t esz = 8;
  cudaStream_t user = nullptr, st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<Level> L;
  Scratch S{};
  void* scratch_mem = nullptr;
  DevScalars* ds = nullptr;
  double* partials = nullptr;
  int n_partials = 0;
  double* ring = nullptr;
  long long* ring_pos = nullptr;
  int ring_cap = 4096;
  double* wsum = nullptr;
  double* stage = nullptr;  // device staging for field I/O
  double* hstage = nullptr; // pinned host staging
  size_t stage_elems = 0;
  Phys P{};
  df_params prm{};
  bool have_params = false;
  int xi[DF_MAX_LEVELS];
  cudaGraphExec_t gexec = nullptr;
  long long graph_kernels = 0;
  long long launches = 0;
  bool timing = false;
  struct EvPair {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<EvPair> evpool;
  size_t ev_used = 0;
  double k_ms[K_NKINDS] = {};
  long long k_n[K_NKINDS] = {};
  int full_boxes = 0;  // 1: every operator on its whole stencil range (debug/parity)
  bool stepped = false;
};

namespace {

// Run one launcher; in timing mode bracket it with a pooled event pair of `kind`.
template <class Fn>
long long timed(df_ctx* c, int kind, Fn&& fn) {
  if (!c->timing) return fn();
  if (c->ev_used == c->evpool.size()) {
    df_ctx::EvPair p;
    cudaEventCreate(&p.a);
    cudaEventCreate(&p.b);
    c->evpool.push_back(p);
  }
  df_ctx::EvPair& p = c->evpool[c->ev_used++];
  p.kind = kind;
  cudaEventRecord(p.a, c->st);
  long long n = fn();
  cudaEventRecord(p.b, c->st);
  return n;
}

// Fold the recorded event pairs into the per-kind totals (synchronises).
void harvest_timing(df_ctx* c) {
  if (!c->ev_used) return;
  cudaStreamSynchronize(c->st);
  for (size_t i = 0; i < c->ev_used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->evpool[i].a, c->evpool[i].b);
    c->k_ms[c->evpool[i].kind] += ms;
    c->k_n[c->evpool[i].kind] += 1;
  }
  c->ev_used = 0;
}

template <class T>
struct Ops {
  // device address of level l's step in T
  static const T* level_dt(df_ctx* c, int l) {
    if (sizeof(T) == 8) return (const T*)&c->ds->dtl[l];
    return (const T*)&c->ds->dtf[l];
  }

  static Box box(const df_ctx* c, const LevelView& v, int margin) {
    Box b;
    int M = c->full_boxes ? v.G : margin;
    for (int d = 0; d < 3; ++d) {
      b.lo[d] = std::max(0, v.G - M);
      b.hi[d] = std::min(v.s[d], v.G + v.n[d] + M);
    }
    return b;
  }

  static long long level_step(df_ctx* c, int l, int m_out) {
    LevelView& v = c->L[l].v;
    const Phys& P = c->P;
    cudaStream_t st = c->st;
    const T* dt = level_dt(c, l);
    const Scratch& S = c->S;
    long long n = 0;
    Box b = box(c, v, m_out + kReach);
    double gm1 = P.gamma - 1.0;
    if (l == 0) n += timed(c, K_BC, [&] { return launch_bc_fill<T>(v, P, st); });
    if (P.hydro_on)
      n += timed(c, K_SOURCE, [&] { return launch_source<T>(v, b, S, dt, 1, gm1, P, st); });
    int do_lum = P.L != 0.0, do_eps = P.chi > 0.0;
    if (P.hydro_on || do_lum || do_eps)
      n += timed(c, K_COMPRESS, [&] {
        return launch_compress_lum<T>(v, b, S, dt, P, P.hydro_on, do_lum, do_eps, st);
      });
    if (P.chi > 0.0) {
      if (v.is_child)
        n += timed(c, K_FRONTIER_DIFF, [&] { return launch_frontier_diff<T>(v, S, dt, P, st); });
      n += timed(c, K_DIFFUSE, [&] { return launch_diffuse<T>(v, b, S, dt, P, st); });
    }
    if (P.hydro_on) {
      for (int d = 0; d < 3; ++d) {
        n += timed(c, K_TPREP, [&] { return launch_tprep<T>(v, b, S, P, st); });
        n += timed(c, K_TFLUX, [&] { return launch_tflux<T>(v, b, S, d, dt, P, st); });
        if (v.is_child)
          n += timed(c, K_TFRONTIER, [&] { return launch_tfrontier<T>(v, S, d, st); });
        n += timed(c, K_TMOM, [&] { return launch_tmom<T>(v, b, S, d, dt, P, st); });
        n += timed(c, K_TUPDATE, [&] { return launch_tupdate<T>(v, b, S, d, st); });
      }
      n += timed(c, K_VREC_SOURCE,
                 [&] { return launch_vrec_source<T>(v, b, S, dt, gm1, P, st); });
    }
    return n;
  }

  static long long advance(df_ctx* c, int l, int m_out) {
    long long n = 0;
    if (l + 1 < c->nl) {
      Level& ch = c->L[l + 1];
      cudaMemsetAsync(ch.acc, 0, ch.acc_elems * sizeof(double), c->st);
      int xi = c->xi[l];
      for (int s = 0; s < xi; ++s) n += advance(c, l + 1, (xi - 1 - s) * kReach);
    }
    n += level_step(c, l, m_out);
    if (l + 1 < c->nl) {
      const LevelView &cv = c->L[l].v, &fv = c->L[l + 1].v;
      n += timed(c, K_COMMUP, [&] { return launch_commup<T>(cv, fv, c->st); });
      n += timed(c, K_COMMMEAN, [&] { return launch_commmean<T>(cv, fv, c->P.band, c->st); });
    }
    return n;
  }

  static void prods(const df_ctx* c, double* out /* 5*nl */) {
    double pr = 1.0;
    for (int l = 0; l < c->nl; ++l) {
      if (l > 0) pr *= c->xi[l - 1];
      out[l] = pr;
      const LevelView& v = c->L[l].v;
      double lim = INFINITY;
      if (c->P.chi > 0.0) {
        double sinv = 0.0;
        for (int d = 0; d < 3; ++d) sinv += 1.0 / (v.dx[d] * v.dx[d]);
        lim = c->P.cfl_diff / (2.0 * c->P.chi * sinv);
      }
      out[c->nl + l] = lim;
      for (int d = 0; d < 3; ++d)
        out[2 * c->nl + 3 * l + d] = c->P.hydro_on ? c->P.cfl * v.dx[d] : 0.0;
    }
  }

  static long long dt_levels(df_ctx* c) {
    long long n = 0;
    for (int l = 0; l < c->nl; ++l)
      n += timed(c, K_DT, [&] { return launch_dt_level<T>(c->L[l].v, l, c->P, c->ds, c->st); });
    return n;
  }

  static long long force(df_ctx* c, bool ring) {
    long long n = 0;
    int off = 0;
    for (int l = 0; l < c->nl; ++l) {
      n += timed(c, K_FORCE,
                 [&] { return launch_force_level<T>(c->L[l].v, c->P, c->partials, off, c->st); });
      off += force_partials_per_level(c->L[l].v);
    }
    n += timed(c, K_FORCE, [&] {
      return launch_force_finalize(c->partials, off, c->ds, ring ? c->ring : nullptr,
                                   c->ring_cap, c->ring_pos, c->st);
    });
    return n;
  }

  // one coarse step with the current xi word
  static long long coarse_step(df_ctx* c) {
    long long n = dt_levels(c);
    double pr[5 * DF_MAX_LEVELS];
    prods(c, pr);
    n += timed(c, K_DT, [&] { return launch_dt_finalize(c->ds, c->nl, pr, c->P.dt_fixed, c->st); });
    n += advance(c, 0, 0);
    n += force(c, true);
    n += timed(c, K_OTHER, [&] { return launch_time_advance(c->ds, c->st); });
    return n;
  }
};

template <class T>
int run_steps(df_ctx* c, int nsteps) {
  if (c->P.dt_fixed <= 0.0 && c->P.hydro_on == 0 && !(c->P.chi > 0.0))
    return fail(DF_EINVAL, "no time-step limit: set dt_fixed, hydro_on or chi");
  if (c->prm.xi_mode == 1 && c->nl > 1) {
    // Eq. 55-56 search each coarse step: per-level limits come back to the host
    for (int s = 0; s < nsteps; ++s) {
      c->launches += Ops<T>::dt_levels(c);
      unsigned long long bits[3 * DF_MAX_LEVELS];
      CK(cudaMemcpyAsync(bits, c->ds->dtmin, 3 * c->nl * sizeof(unsigned long long),
                         cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      double pr[5 * DF_MAX_LEVELS], lim[DF_MAX_LEVELS], cost[DF_MAX_LEVELS];
      for (int l = 0; l < c->nl; ++l) c->xi[l] = 2;
      Ops<T>::prods(c, pr);
      for (int l = 0; l < c->nl; ++l) {
        lim[l] = pr[c->nl + l];
        for (int d = 0; d < 3; ++d) {
          double mx;
          memcpy(&mx, &bits[3 * l + d], 8);
          lim[l] = std::min(lim[l], pr[2 * c->nl + 3 * l + d] / mx);
        }
        cost[l] = (double)c->n[0] * c->n[1] * c->n[2];
      }
      int xiw[DF_MAX_LEVELS];
      double ratio;
      df_xi_search(c->nl, lim, cost, xiw, &ratio);
      for (int l = 0; l + 1 < c->nl; ++l) c->xi[l] = xiw[l];
      Ops<T>::prods(c, pr);
      long long n = launch_dt_finalize(c->ds, c->nl, pr, c->P.dt_fixed, c->st);
      n += Ops<T>::advance(c, 0, 0);
      n += Ops<T>::force(c, true);
      n += launch_time_advance(c->ds, c->st);
      c->launches += n;
    }
    CK(cudaGetLastError());
    return DF_OK;
  }
  for (int l = 0; l < c->nl; ++l) c->xi[l] = 2;
  if (c->timing) {
    for (int s = 0; s < nsteps; ++s) c->launches += Ops<T>::coarse_step(c);
    CK(cudaGetLastError());
    return DF_OK;
  }
  if (!c->gexec) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
    long long n = Ops<T>::coarse_step(c);
    cudaError_t e = cudaStreamEndCapture(c->st, &g);
    if (e != cudaSuccess) return fail(DF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(DF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->graph_kernels = n;
  }
  for (int s = 0; s < nsteps; ++s) {
    CK(cudaGraphLaunch(c->gexec, c->st));
    c->launches += c->graph_kernels;
  }
  return DF_OK;
}

int check_ctx(df_ctx* c, bool need_params = true) {
  if (!c) return fail(DF_EINVAL, "null context");
  if (need_params && !c->have_params) return fail(DF_EINVAL, "df_set_params not called");
  return DF_OK;
}

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

void enter(df_ctx* c) {
  cudaEventRecord(c->ev_in, c->user);
  cudaStreamWaitEvent(c->st, c->ev_in, 0);
}
void leave(df_ctx* c) {
  cudaEventRecord(c->ev_out, c->st);
  cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

int sync_health(df_ctx* c) {
  CK(cudaStreamSynchronize(c->st));
  int bad = 0;
  CK(cudaMemcpy(&bad, &c->ds->unhealthy, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) return fail(DF_EUNHEALTHY, "NaN, rho <= 0 or e <= 0 found in the state");
  return DF_OK;
}

// background value of a field (the stored state is the deviation from it)
double field_bg(const df_ctx* c, int field) {
  return field == 0 ? c->P.rho0 : field == 1 ? c->P.e0 : c->P.V[field - 2];
}

template <class T>
int do_io(df_ctx* c, int level, int field, double* out, const double* in, int full,
          bool raw = false) {
  if (level < 0 || level >= c->nl || field < 0 || field > 4)
    return fail(DF_EINVAL, "level %d / field %d out of range", level, field);
  LevelView& v = c->L[level].v;
  size_t n = full ? (size_t)v.nc : (size_t)v.n[0] * v.n[1] * v.n[2];
  if (in) {
    CK(cudaMemcpyAsync(c->stage, in, n * sizeof(double), cudaMemcpyHostToDevice, c->st));
    double bgv = raw ? 0.0 : field_bg(c, field);
    c->launches += launch_unpack_active<T>(v, field, c->stage, full, bgv, c->st);
  } else {
    double bgv = raw ? 0.0 : field_bg(c, field);
    c->launches += launch_pack_active<T>(v, field, c->stage, full, bgv, c->st);
    CK(cudaMemcpyAsync(out, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  return DF_OK;
}

void free_ctx(df_ctx* c) {
  if (!c) return;
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (auto& l : c->L) {
    cudaFree(l.mem);
    cudaFree(l.acc);
    cudaFree(l.v.fw);
  }
  cudaFree(c->scratch_mem);
  cudaFree(c->ds);
  cudaFree(c->partials);
  cudaFree(c->ring);
  cudaFree(c->ring_pos);
  cudaFree(c->wsum);
  cudaFree(c->stage);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  for (auto& p : c->evpool) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  if (c->st) cudaStreamDestroy(c->st);
  delete c;
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char* df_last_error(void) { return g_err.c_str(); }

int df_xi_search(int n, const double* dtl, const double* cost, int* xi_out, double* ratio) {
  if (n < 1 || n > DF_MAX_LEVELS || !dtl || !cost) return fail(DF_EINVAL, "bad xi search input");
  double best = -1.0;
  int nw = n - 1;
  for (long w = 0; w < (1L << nw); ++w) {
    double dt = INFINITY, C = 0.0, pr = 1.0;
    for (int l = 0; l < n; ++l) {
      if (l > 0) pr *= ((w >> (l - 1)) & 1) ? 2.0 : 1.0;
      dt = std::min(dt, dtl[l] * pr);  // Eq. 55
      C += cost[l] * pr;               // Eq. 56
    }
    if (dt / C > best) {
      best = dt / C;
      if (xi_out)
        for (int l = 0; l < nw; ++l) xi_out[l] = ((w >> l) & 1) ? 2 : 1;
    }
  }
  if (ratio) *ratio = best;
  return DF_OK;
}

int df_create(df_ctx** out, int n_levels, const int n[3], const double lo[3], const double hi[3],
              int G, int precision, int device, void* stream) {
  if (!out || !n || !lo || !hi) return fail(DF_EINVAL, "null argument");
  *out = nullptr;
  if (n_levels < 1 || n_levels > DF_MAX_LEVELS) return fail(DF_EINVAL, "n_levels out of range");
  if (G < 2 || G % 2) return fail(DF_EINVAL, "G must be even and >= 2");
  if (precision != DF_FP64 && precision != DF_FP32_STATE)
    return fail(DF_EINVAL, "unknown precision %d", precision);
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 8 || n[d] % 4 || n[d] < G) return fail(DF_EINVAL, "n[%d]=%d: need n%%4==0, n>=8, n>=G", d, n[d]);
    if (!(hi[d] > lo[d])) return fail(DF_EINVAL, "empty box on axis %d", d);
  }
  long long s3 = 1;
  for (int d = 0; d < 3; ++d) s3 *= (n[d] + 2 * G);
  if (s3 >= (1LL << 31) / 5) return fail(DF_EINVAL, "level too large (%lld elements)", s3);
  CK(cudaSetDevice(device));
  df_ctx* c = new (std::nothrow) df_ctx;
  if (!c) return fail(DF_ENOMEM, "host allocation");
  c->nl = n_levels;
  c->prec = precision;
  c->device = device;
  c->G = G;
  c->esz = precision == DF_FP64 ? 8 : 4;
  c->user = (cudaStream_t)stream;
  for (int d = 0; d < 3; ++d) {
    c->n[d] = n[d];
    c->lo[d] = lo[d];
    c->hi[d] = hi[d];
  }
  for (int l = 0; l < DF_MAX_LEVELS; ++l) c->xi[l] = 2;
#define CKF(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      int r_ = fail(e_ == cudaErrorMemoryAllocation ? DF_ENOMEM : DF_ECUDA,  \
                    "%s failed: %s", #call, cudaGetErrorString(e_));         \
      free_ctx(c);                                                           \
      return r_;                                                             \
    }                                                                        \
  } while (0)
  CKF(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
  CKF(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
  CKF(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
  c->L.resize(n_levels);
  size_t nc = (size_t)s3;
  for (int l = 0; l < n_levels; ++l) {
    LevelView& v = c->L[l].v;
    memset(&v, 0, sizeof v);
    double scale = std::ldexp(1.0, -l);
    v.G = G;
    v.nc = (int)nc;
    for (int d = 0; d < 3; ++d) {
      v.n[d] = n[d];
      v.s[d] = n[d] + 2 * G;
      v.lo[d] = lo[d] * scale;
      v.dx[d] = (hi[d] - lo[d]) * scale / n[d];
    }
    v.st[0] = 1;
    v.st[1] = v.s[0];
    v.st[2] = v.s[0] * v.s[1];
    v.vol = v.dx[0] * v.dx[1] * v.dx[2];
    v.area[0] = v.dx[1] * v.dx[2];
    v.area[1] = v.dx[0] * v.dx[2];
    v.area[2] = v.dx[0] * v.dx[1];
    v.inv_vol = 1.0 / v.vol;
    for (int d = 0; d < 3; ++d) {
      v.inv_dx[d] = 1.0 / v.dx[d];
      v.dcoef[d] = v.area[d] / v.dx[d];
    }
    v.dt_scale = scale;
    v.is_child = l > 0;
    if (l > 0) {
      const LevelView& p = c->L[l - 1].v;
      for (int d = 0; d < 3; ++d) {
        double o = (v.lo[d] - p.lo[d]) / p.dx[d];
        int oi = (int)std::floor(o + 0.5);
        if (std::fabs(o - oi) > 1e-9 || oi < G / 2 + 1 || oi + n[d] / 2 + G / 2 + 1 > p.n[d]) {
          int r = fail(DF_EINVAL,
                       "level %d: offset %.3f on axis %d must be an integer in [%d, %d]", l, o,
                       d, G / 2 + 1, p.n[d] - n[d] / 2 - G / 2 - 1);
          free_ctx(c);
          return r;
        }
        v.off[d] = oi;
      }
    }
    // one allocation: 5 fields + potential + luminosity weights, 256-B aligned planes
    size_t plane = ((nc * c->esz + 255) / 256) * 256;
    CKF(cudaMalloc(&c->L[l].mem, plane * 7));
    char* base = (char*)c->L[l].mem;
    for (int f = 0; f < 5; ++f) v.q[f] = base + plane * f;
    v.phi = base + plane * 5;
    v.lumw = base + plane * 6;
    // frontier accumulators (this level as a child): 6 sides x 3 quantities
    int slots = 0;
    for (int d = 0; d < 3; ++d) {
      int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      slots = std::max(slots, (n[t1] / 2) * (n[t2] / 2));
    }
    v.acc_slots = slots;
    c->L[l].acc_elems = (size_t)18 * slots;
    CKF(cudaMalloc(&c->L[l].acc, c->L[l].acc_elems * sizeof(double)));
    CKF(cudaMalloc(&v.fw, (size_t)n[0] * n[1] * n[2] * sizeof(double)));
    CKF(cudaMemset(c->L[l].acc, 0, c->L[l].acc_elems * sizeof(double)));
    v.acc = c->L[l].acc;
  }
  for (int l = 0; l + 1 < n_levels; ++l) {
    LevelView& v = c->L[l].v;
    const LevelView& ch = c->L[l + 1].v;
    v.has_child = 1;
    for (int d = 0; d < 3; ++d) {
      v.coff[d] = ch.off[d];
      v.cn[d] = ch.n[d];
    }
    v.cacc = ch.acc;
    v.cacc_slots = ch.acc_slots;
  }
  // shared scratch: pi[3], eps, w[3], F, E, P[3]
  size_t plane = ((nc * c->esz + 255) / 256) * 256;
  CKF(cudaMalloc(&c->scratch_mem, plane * 12));
  CKF(cudaMemset(c->scratch_mem, 0, plane * 12));
  {
    char* b = (char*)c->scratch_mem;
    for (int m = 0; m < 3; ++m) c->S.pi[m] = b + plane * m;
    c->S.eps = b + plane * 3;
    for (int m = 0; m < 3; ++m) c->S.w[m] = b + plane * (4 + m);
    c->S.F = b + plane * 7;
    c->S.E = b + plane * 8;
    for (int m = 0; m < 3; ++m) c->S.P[m] = b + plane * (9 + m);
  }
  CKF(cudaMalloc(&c->ds, sizeof(DevScalars)));
  CKF(cudaMemset(c->ds, 0, sizeof(DevScalars)));
  // partials: 3 per force block of every level, and one per 256 active cells of a
  // level for the luminosity normalisation (the two uses never overlap in time)
  int np = 0;
  for (int l = 0; l < n_levels; ++l) np += force_partials_per_level(c->L[l].v);
  c->n_partials = np;
  size_t lum_blocks = ((size_t)n[0] * n[1] * n[2] + 255) / 256;
  size_t pelems = std::max(3 * (size_t)np, lum_blocks);
  CKF(cudaMalloc(&c->partials, pelems * sizeof(double)));
  CKF(cudaMalloc(&c->ring, 3 * (size_t)c->ring_cap * sizeof(double)));
  CKF(cudaMalloc(&c->ring_pos, sizeof(long long)));
  CKF(cudaMemset(c->ring_pos, 0, sizeof(long long)));
  CKF(cudaMalloc(&c->wsum, sizeof(double)));
  c->stage_elems = nc;
  CKF(cudaMalloc(&c->stage, nc * sizeof(double)));
#undef CKF
  *out = c;
  return DF_OK;
}

int df_set_params(df_ctx* c, const df_params* p) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!p) return fail(DF_EINVAL, "null params");
  if (!(p->gamma > 1.0) || !(p->rho0 > 0.0) || !(p->cs > 0.0) || p->chi < 0.0 ||
      !(p->cfl > 0.0) || p->band < 1 || p->mach < 0.0)
    return fail(DF_EINVAL, "invalid physical parameters");
  if (p->chi > 0.0 && !(p->cfl_diff > 0.0)) return fail(DF_EINVAL, "cfl_diff must be > 0");
  for (int k = 0; k < 6; ++k)
    if (p->bc[k] < 0 || p->bc[k] > 3) return fail(DF_EINVAL, "bad boundary type");
  DevGuard g(c->device);
  c->prm = *p;
  Phys& P = c->P;
  P.gamma = p->gamma;
  P.rho0 = p->rho0;
  P.e0 = p->cs * p->cs * p->rho0 / (p->gamma * (p->gamma - 1.0));  // Sec. 3.4
  for (int d = 0; d < 3; ++d) P.V[d] = p->mach * p->cs * p->flow_dir[d];
  P.GM = p->GM;
  P.eps = p->eps;
  P.chi = p->chi;
  P.L = p->L;
  P.cfl = p->cfl;
  P.cfl_diff = p->cfl_diff;
  P.dt_fixed = p->dt_fixed;
  P.diff_face_rho = p->diff_face_rho;
  P.hydro_on = p->hydro_on;
  P.band = p->band;
  for (int k = 0; k < 6; ++k) P.bc[k] = p->bc[k];
  enter(c);
  for (int l = 0; l < c->nl; ++l) {
    LevelView& v = c->L[l].v;
    c->launches += c->prec == DF_FP64 ? launch_init_uniform<double>(v, P, c->st)
                                      : launch_init_uniform<float>(v, P, c->st);
    if (c->prec == DF_FP64) {
      c->launches += launch_static_fields<double>(v, P, p->lum_sigma, c->wsum, c->partials, c->st);
      if (p->lum_sigma > 0.0) c->launches += launch_normalise_lum<double>(v, c->wsum, c->st);
    } else {
      c->launches += launch_static_fields<float>(v, P, p->lum_sigma, c->wsum, c->partials, c->st);
      if (p->lum_sigma > 0.0) c->launches += launch_normalise_lum<float>(v, c->wsum, c->st);
    }
    CK(cudaMemsetAsync(c->L[l].acc, 0, c->L[l].acc_elems * sizeof(double), c->st));
    c->launches += launch_force_weights(v, P, c->st);
  }
  DevScalars h;
  memset(&h, 0, sizeof h);
  // per-axis maxima start at +0.0 (bit pattern 0)
  CK(cudaMemcpyAsync(c->ds, &h, sizeof h, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->ring_pos, 0, sizeof(long long), c->st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  c->have_params = true;
  c->stepped = false;
  return DF_OK;
}

int df_step(df_ctx* c, int n) {
  if (check_ctx(c)) return DF_EINVAL;
  if (n < 0) return fail(DF_EINVAL, "negative step count");
  if (n == 0) return DF_OK;
  DevGuard g(c->device);
  enter(c);
  int r = c->prec == DF_FP64 ? run_steps<double>(c, n) : run_steps<float>(c, n);
  leave(c);
  c->stepped = true;
  return r;
}

int df_status(df_ctx* c, double* t, double* dt_last, int* unhealthy) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  CK(cudaStreamSynchronize(c->st));
  DevScalars h;
  CK(cudaMemcpy(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost));
  if (t) *t = h.t;
  if (dt_last) *dt_last = h.dt;
  if (unhealthy) *unhealthy = h.unhealthy;
  return DF_OK;
}

int df_force_now(df_ctx* c, double F[3]) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!F) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  enter(c);
  c->launches += c->prec == DF_FP64 ? Ops<double>::force(c, false) : Ops<float>::force(c, false);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  DevScalars h;
  CK(cudaMemcpy(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost));
  for (int d = 0; d < 3; ++d) F[d] = h.F[d];
  return DF_OK;
}

int df_force(df_ctx* c, double F[3], double* along) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!F) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  int r;
  if (!c->stepped) {
    r = df_force_now(c, F);
    if (r) return r;
  } else {
    r = sync_health(c);
    DevScalars h;
    CK(cudaMemcpy(&h, c->ds, sizeof h, cudaMemcpyDeviceToHost));
    for (int d = 0; d < 3; ++d) F[d] = h.F[d];
    if (r) return r;
  }
  if (along) {
    double nv = std::sqrt(c->P.V[0] * c->P.V[0] + c->P.V[1] * c->P.V[1] + c->P.V[2] * c->P.V[2]);
    *along = nv > 0 ? -(F[0] * c->P.V[0] + F[1] * c->P.V[1] + F[2] * c->P.V[2]) / nv : 0.0;
  }
  return DF_OK;
}

int df_compute_dt(df_ctx* c, double* dt, double* dt_level) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  enter(c);
  long long n =
      c->prec == DF_FP64 ? Ops<double>::dt_levels(c) : Ops<float>::dt_levels(c);
  double pr[5 * DF_MAX_LEVELS];
  for (int l = 0; l < c->nl; ++l) c->xi[l] = 2;
  if (c->prec == DF_FP64)
    Ops<double>::prods(c, pr);
  else
    Ops<float>::prods(c, pr);
  // the finalize kernel overwrites the coarse step; keep the last one taken
  DevScalars before;
  CK(cudaMemcpyAsync(&before, c->ds, sizeof before, cudaMemcpyDeviceToHost, c->st));
  n += launch_dt_finalize(c->ds, c->nl, pr, c->P.dt_fixed, c->st);
  DevScalars after;
  CK(cudaMemcpyAsync(&after, c->ds, sizeof after, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemcpyAsync(&c->ds->dt, &before.dt, sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  c->launches += n;
  if (dt) *dt = after.dt;
  if (dt_level)
    for (int l = 0; l < c->nl; ++l) dt_level[l] = after.dtlev[l];
  return DF_OK;
}

int df_get_field(df_ctx* c, int level, int field, double* out) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  enter(c);
  int r = c->prec == DF_FP64 ? do_io<double>(c, level, field, out, nullptr, 0)
                             : do_io<float>(c, level, field, out, nullptr, 0);
  leave(c);
  return r;
}

int df_set_field(df_ctx* c, int level, int field, const double* in) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  DevGuard g(c->device);
  enter(c);
  int r = c->prec == DF_FP64 ? do_io<double>(c, level, field, nullptr, in, 0)
                             : do_io<float>(c, level, field, nullptr, in, 0);
  leave(c);
  return r;
}

int df_get_full(df_ctx* c, int level, int field, double* out) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  enter(c);
  int r = c->prec == DF_FP64 ? do_io<double>(c, level, field, out, nullptr, 1)
                             : do_io<float>(c, level, field, out, nullptr, 1);
  leave(c);
  return r;
}

int df_set_full(df_ctx* c, int level, int field, const double* in) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  DevGuard g(c->device);
  enter(c);
  int r = c->prec == DF_FP64 ? do_io<double>(c, level, field, nullptr, in, 1)
                             : do_io<float>(c, level, field, nullptr, in, 1);
  leave(c);
  return r;
}

size_t df_state_size(const df_ctx* c) {
  if (!c) return 0;
  return (size_t)c->nl * 5 * (size_t)c->L[0].v.nc;
}

int df_get_state(df_ctx* c, double* out, double* t_out) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  size_t nc = (size_t)c->L[0].v.nc;
  DevGuard g(c->device);
  enter(c);
  for (int l = 0; l < c->nl; ++l)
    for (int f = 0; f < 5; ++f) {
      int r = c->prec == DF_FP64
                  ? do_io<double>(c, l, f, out + (l * 5 + f) * nc, nullptr, 1, true)
                  : do_io<float>(c, l, f, out + (l * 5 + f) * nc, nullptr, 1, true);
      if (r) return r;
    }
  leave(c);
  if (t_out) return df_status(c, t_out, nullptr, nullptr);
  return DF_OK;
}

int df_set_state(df_ctx* c, const double* in, double t) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  size_t nc = (size_t)c->L[0].v.nc;
  DevGuard g(c->device);
  enter(c);
  for (int l = 0; l < c->nl; ++l)
    for (int f = 0; f < 5; ++f) {
      int r = c->prec == DF_FP64
                  ? do_io<double>(c, l, f, nullptr, in + (l * 5 + f) * nc, 1, true)
                  : do_io<float>(c, l, f, nullptr, in + (l * 5 + f) * nc, 1, true);
      if (r) return r;
    }
  leave(c);
  CK(cudaMemcpy(&c->ds->t, &t, sizeof(double), cudaMemcpyHostToDevice));
  int zero = 0;
  CK(cudaMemcpy(&c->ds->unhealthy, &zero, sizeof(int), cudaMemcpyHostToDevice));
  c->stepped = false;
  return DF_OK;
}

int df_prolong(df_ctx* c, int cl) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (cl < 0 || cl + 1 >= c->nl) return fail(DF_EINVAL, "no level below %d", cl);
  DevGuard g(c->device);
  enter(c);
  c->launches += c->prec == DF_FP64 ? launch_commup<double>(c->L[cl].v, c->L[cl + 1].v, c->st)
                                    : launch_commup<float>(c->L[cl].v, c->L[cl + 1].v, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  return DF_OK;
}

int df_restrict(df_ctx* c, int cl) {
  if (check_ctx(c)) return DF_EINVAL;
  if (cl < 0 || cl + 1 >= c->nl) return fail(DF_EINVAL, "no level below %d", cl);
  DevGuard g(c->device);
  enter(c);
  c->launches += c->prec == DF_FP64
                     ? launch_commmean<double>(c->L[cl].v, c->L[cl + 1].v, c->P.band, c->st)
                     : launch_commmean<float>(c->L[cl].v, c->L[cl + 1].v, c->P.band, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  return DF_OK;
}

int df_fill_bc(df_ctx* c) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  enter(c);
  c->launches += c->prec == DF_FP64 ? launch_bc_fill<double>(c->L[0].v, c->P, c->st)
                                    : launch_bc_fill<float>(c->L[0].v, c->P, c->st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  leave(c);
  return DF_OK;
}

long long df_kernel_launches(const df_ctx* c) { return c ? c->launches : -1; }

int df_set_timing(df_ctx* c, int on) {
  if (!c) return fail(DF_EINVAL, "null context");
  DevGuard g(c->device);
  harvest_timing(c);
  c->timing = on != 0;
  for (int k = 0; k < K_NKINDS; ++k) {
    c->k_ms[k] = 0.0;
    c->k_n[k] = 0;
  }
  return DF_OK;
}

int df_kernel_time(df_ctx* c, int kind, double* ms, long long* launches) {
  if (!c || kind < 0 || kind >= K_NKINDS) return fail(DF_EINVAL, "bad timing query");
  DevGuard g(c->device);
  harvest_timing(c);
  if (ms) *ms = c->k_ms[kind];
  if (launches) *launches = c->k_n[kind];
  return DF_OK;
}

const char* df_kernel_name(int kind) {
  static const char* names[K_NKINDS] = {
      "bc_fill",  "source",   "compress_lum", "diffuse",  "frontier_diff", "tprep",
      "tflux",    "tfrontier", "tmom",        "tupdate",  "vrec_source",   "commup",
      "commmean", "dt",       "force",        "other"};
  return kind >= 0 && kind < K_NKINDS ? names[kind] : "";
}

int df_debug_full_boxes(df_ctx* c, int on) {
  if (!c) return fail(DF_EINVAL, "null context");
  c->full_boxes = on != 0;
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
  return DF_OK;
}

int df_check_division(const double* a_host, const double* b_host, int n, double* max_ulp) {
  if (!a_host || !b_host || !max_ulp || n < 1) return fail(DF_EINVAL, "bad division check input");
  double *da = nullptr, *db = nullptr, *dm = nullptr;
  CK(cudaMalloc(&da, n * sizeof(double)));
  CK(cudaMalloc(&db, n * sizeof(double)));
  CK(cudaMalloc(&dm, sizeof(double)));
  CK(cudaMemcpy(da, a_host, n * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(db, b_host, n * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemset(dm, 0, sizeof(double)));
  launch_hdiv_check(da, db, n, dm, nullptr);
  CK(cudaGetLastError());
  CK(cudaMemcpy(max_ulp, dm, sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(da);
  cudaFree(db);
  cudaFree(dm);
  return DF_OK;
}

int df_destroy(df_ctx* c) {
  if (!c) return DF_OK;
  DevGuard g(c->device);
  cudaStreamSynchronize(c->st);
  free_ctx(c);
  return DF_OK;
}

}  // extern "C"
