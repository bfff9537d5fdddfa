// dfnest.cu -- host runtime and C ABI of libdfnest.so (see include/dfnest.h).
//
// A *run* is one hierarchy of Sec. 3 resident on one GPU: one padded allocation of
// 7 planes per level (5 fields, potential, luminosity weights), a scratch set
// shared by its levels (they are advanced one at a time), frontier slabs, force
// weights, and device scalars (time step, time, force, health flag).
//
// A *plan* is the launch list of one coarse step of a set of runs: the Eq. 55 time
// step, the recursion of Sec. 3.3 and the Eq. 18 force of every run, as work items
// of the persistent work-list kernel (kernels.cu).  The op lists of the runs are
// merged so that one launch carries the same op for every run that has it next;
// the plan is uploaded once and captured into a CUDA graph, and the time step is
// read by the kernels from device memory, so stepping never synchronises the host.
// A context (df_ctx) is one run and its plan; a pool (df_pool) is many runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
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
      return fail(e_ == cudaErrorMemoryAllocation ? DF_ENOMEM : DF_ECUDA,            \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                   \
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

namespace {

// ------------------------------------------------------------------ device memory

// Where a context's or pool's device memory comes from: cudaMalloc / cudaFree, or
// the caller's allocator (df_set_allocator), captured when the owner is created.
struct Allocator {
  df_alloc_fn alloc = nullptr;
  df_free_fn dealloc = nullptr;
  void* user = nullptr;
};
Allocator g_allocator;  // applies to owners created from now on

cudaError_t dev_alloc(const Allocator& a, void** p, size_t bytes) {
  if (!a.alloc) return cudaMalloc(p, bytes);
  *p = a.alloc(bytes, a.user);
  if (!*p) return cudaErrorMemoryAllocation;
  if ((uintptr_t)*p % 256) {  // the kernels' planes and vector loads assume it
    a.dealloc(*p, a.user);
    *p = nullptr;
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

void dev_free(const Allocator& a, void* p) {
  if (!p) return;
  if (!a.alloc)
    cudaFree(p);
  else
    a.dealloc(p, a.user);
}

// ------------------------------------------------------------------------- runs

struct Run {
  int nl = 0, prec = 0, G = 0;
  int n0[3] = {0, 0, 0};  // cells per axis of the ground level
  int n[3] = {0, 0, 0};   // of every finer level
  size_t nc_max = 0;      // elements per field of the largest level
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  size_t esz = 8;
  Allocator al;  // every device buffer of the run
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
  Phys P{};
  df_params prm{};
  bool have_params = false;
  bool stepped = false;
  int xi[DF_MAX_LEVELS];
  size_t bytes = 0;
};

size_t plane_bytes(size_t nc, size_t esz) { return ((nc * esz + 255) / 256) * 256; }

// cells per axis of level l: the ground's own counts, then the finer levels'
inline const int* level_n(int l, const int n0[3], const int n[3]) { return l == 0 ? n0 : n; }

// level l's box is the ground's scaled about the origin by this factor along d: the
// cell halves from level to level (n0 == n: 2^-l; n0 == 2n: level 1 spans a quarter)
inline double level_scale(int l, int d, const int n0[3], const int n[3]) {
  return std::ldexp((double)level_n(l, n0, n)[d] / n0[d], -l);
}

size_t level_elems(const int n[3], int G) {
  size_t nc = 1;
  for (int d = 0; d < 3; ++d) nc *= (size_t)(n[d] + 2 * G);
  return nc;
}

// device bytes a run of this shape allocates (admission control uses the same sum)
size_t run_bytes(int nl, const int n0[3], const int n[3], int G, int prec) {
  size_t esz = prec == DF_FP64 ? 8 : 4;
  size_t total = 0, nc_max = 0, na_max = 0, np = 0;
  for (int l = 0; l < nl; ++l) {
    const int* m = level_n(l, n0, n);
    size_t nc = level_elems(m, G), na = (size_t)m[0] * m[1] * m[2];
    const int sp[3] = {m[0] + 2 * G, m[1] + 2 * G, m[2] + 2 * G};
    int slots = 0;
    for (int d = 0; d < 3; ++d) {
      int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      slots = std::max(slots, (m[t1] / 2) * (m[t2] / 2));
    }
    total += plane_bytes(nc, esz) * 7 + ((size_t)rec_elems(sp) + 18 * (size_t)slots) * 8 +
             3 * na * 8;
    np += (na + 2047) / 2048;
    nc_max = std::max(nc_max, nc);
    na_max = std::max(na_max, na);
  }
  size_t pel = std::max(3 * np, (na_max + 255) / 256);
  return total + plane_bytes(nc_max, esz) * 12 + sizeof(DevScalars) + pel * 8 +
         kRingStride * 4096 * 8 + 8 + 8 + nc_max * 8;
}

void run_free(Run* r) {
  if (!r) return;
  const Allocator& a = r->al;
  for (auto& l : r->L) {
    dev_free(a, l.mem);
    dev_free(a, l.acc);
    dev_free(a, l.v.fw);
  }
  dev_free(a, r->scratch_mem);
  dev_free(a, r->ds);
  dev_free(a, r->partials);
  dev_free(a, r->ring);
  dev_free(a, r->ring_pos);
  dev_free(a, r->wsum);
  dev_free(a, r->stage);
  delete r;
}

int check_shape(int n_levels, const int n0[3], const int n[3], const double lo[3],
                const double hi[3], int G, int precision) {
  if (n_levels < 1 || n_levels > DF_MAX_LEVELS) return fail(DF_EINVAL, "n_levels out of range");
  if (G < 2 || G % 2) return fail(DF_EINVAL, "G must be even and >= 2");
  if (precision != DF_FP64 && precision != DF_FP32_STATE)
    return fail(DF_EINVAL, "unknown precision %d", precision);
  for (int l = 0; l < std::min(n_levels, 2); ++l) {
    const int* m = level_n(l, n0, n);
    for (int d = 0; d < 3; ++d)
      if (m[d] < 8 || m[d] % 4 || m[d] < G)
        return fail(DF_EINVAL, "level %d: n[%d]=%d: need n%%4==0, n>=8, n>=G", l, d, m[d]);
    long long s3 = 1;
    for (int d = 0; d < 3; ++d) s3 *= (m[d] + 2 * G);
    if (s3 >= (1LL << 31) / 5)
      return fail(DF_EINVAL, "level %d too large (%lld elements)", l, s3);
  }
  for (int d = 0; d < 3; ++d)
    if (!(hi[d] > lo[d])) return fail(DF_EINVAL, "empty box on axis %d", d);
  // every finer level on parent faces, ghosts and CommUp stencil inside the parent;
  // a lower domain face at coordinate 0 keeps every level on it (offset 0), which
  // df_set_params accepts only when that face is a mirror plane
  for (int l = 1; l < n_levels; ++l)
    for (int d = 0; d < 3; ++d) {
      const int pn = level_n(l - 1, n0, n)[d], cn = n[d];
      double ps = level_scale(l - 1, d, n0, n), cs = level_scale(l, d, n0, n);
      double plo = lo[d] * ps, pdx = (hi[d] - lo[d]) * ps / pn;
      double o = (lo[d] * cs - plo) / pdx;
      int oi = (int)std::floor(o + 0.5);
      bool lo_ok = lo[d] == 0.0 ? oi == 0 : oi >= G / 2 + 1;
      if (std::fabs(o - oi) > 1e-9 || !lo_ok || oi + cn / 2 + G / 2 + 1 > pn)
        return fail(DF_EINVAL, "level %d: offset %.3f on axis %d must be an integer in [%d, %d]",
                    l, o, d, lo[d] == 0.0 ? 0 : G / 2 + 1, pn - cn / 2 - G / 2 - 1);
    }
  return DF_OK;
}

// mirror planes: bit d set when the lower d-face lies at coordinate 0 and reflects
int mirror_mask(const double lo[3], const df_params* p) {
  int m = 0;
  for (int d = 0; d < 3; ++d)
    if (lo[d] == 0.0 && p->bc[2 * d] == DF_BC_REFLECT) m |= 1 << d;
  return m;
}

// finer levels may only sit on the domain's lower face across a mirror plane
int check_mirror(int n_levels, const double lo[3], const df_params* p) {
  if (n_levels < 2) return DF_OK;
  int m = mirror_mask(lo, p);
  for (int d = 0; d < 3; ++d)
    if (lo[d] == 0.0 && !(m >> d & 1))
      return fail(DF_EINVAL,
                  "axis %d: finer levels start on the lower face, which must then reflect", d);
  return DF_OK;
}

int run_create(Run** out, int n_levels, const int n0[3], const int n[3], const double lo[3],
               const double hi[3], int G, int precision, const Allocator& al) {
  *out = nullptr;
  int rc0 = check_shape(n_levels, n0, n, lo, hi, G, precision);
  if (rc0) return rc0;
  Run* r = new (std::nothrow) Run;
  if (!r) return fail(DF_ENOMEM, "host allocation");
  r->nl = n_levels;
  r->prec = precision;
  r->G = G;
  r->al = al;
  r->esz = precision == DF_FP64 ? 8 : 4;
  for (int d = 0; d < 3; ++d) {
    r->n0[d] = n0[d];
    r->n[d] = n[d];
    r->lo[d] = lo[d];
    r->hi[d] = hi[d];
  }
  for (int l = 0; l < DF_MAX_LEVELS; ++l) r->xi[l] = 2;
  r->bytes = run_bytes(n_levels, n0, n, G, precision);
#define CKR(call)                                                            \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      int rc_ = fail(e_ == cudaErrorMemoryAllocation ? DF_ENOMEM : DF_ECUDA, \
                     "%s failed: %s", #call, cudaGetErrorString(e_));        \
      run_free(r);                                                           \
      return rc_;                                                            \
    }                                                                        \
  } while (0)
  r->L.resize(n_levels);
  size_t na_max = 0;
  for (int l = 0; l < n_levels; ++l) {
    const int* m = level_n(l, n0, n);
    r->nc_max = std::max(r->nc_max, level_elems(m, G));
    na_max = std::max(na_max, (size_t)m[0] * m[1] * m[2]);
  }
  for (int l = 0; l < n_levels; ++l) {
    LevelView& v = r->L[l].v;
    memset(&v, 0, sizeof v);
    const int* n = level_n(l, n0, r->n);
    const size_t nc = level_elems(n, G), na = (size_t)n[0] * n[1] * n[2];
    const size_t plane = plane_bytes(nc, r->esz);
    v.G = G;
    v.nc = (int)nc;
    for (int d = 0; d < 3; ++d) {
      const double scale = level_scale(l, d, n0, r->n);
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
    v.dt_scale = std::ldexp(1.0, -l);
    v.is_child = l > 0;
    if (l > 0) {
      const LevelView& p = r->L[l - 1].v;
      for (int d = 0; d < 3; ++d) v.off[d] = (int)std::floor((v.lo[d] - p.lo[d]) / p.dx[d] + 0.5);
    }
    CKR(dev_alloc(r->al, &r->L[l].mem, plane * 7));
    char* base = (char*)r->L[l].mem;
    for (int f = 0; f < 5; ++f) v.q[f] = base + plane * f;
    v.phi = base + plane * 5;
    v.lumw = base + plane * 6;
    int slots = 0;
    for (int d = 0; d < 3; ++d) {
      int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      slots = std::max(slots, (n[t1] / 2) * (n[t2] / 2));
    }
    v.acc_slots = slots;
    r->L[l].acc_elems = (size_t)rec_elems(v.s) + (size_t)18 * slots;
    CKR(dev_alloc(r->al, (void**)&r->L[l].acc, r->L[l].acc_elems * sizeof(double)));
    CKR(cudaMemset(r->L[l].acc, 0, r->L[l].acc_elems * sizeof(double)));
    v.acc = r->L[l].acc;
    CKR(dev_alloc(r->al, (void**)&v.fw, 3 * na * sizeof(double)));
  }
  for (int l = 0; l + 1 < n_levels; ++l) {
    LevelView& v = r->L[l].v;
    const LevelView& ch = r->L[l + 1].v;
    v.has_child = 1;
    for (int d = 0; d < 3; ++d) {
      v.coff[d] = ch.off[d];
      v.cn[d] = ch.n[d];
    }
    v.crec = ch.acc;
    v.csum = ch.acc + rec_elems(ch.s);
    v.cacc = v.csum;
    v.cacc_slots = ch.acc_slots;
  }
  // scratch is shared by the levels (advanced one at a time): sized for the largest
  const size_t plane = plane_bytes(r->nc_max, r->esz);
  CKR(dev_alloc(r->al, &r->scratch_mem, plane * 12));
  CKR(cudaMemset(r->scratch_mem, 0, plane * 12));
  {
    char* b = (char*)r->scratch_mem;
    for (int m = 0; m < 3; ++m) r->S.pi[m] = b + plane * m;
    r->S.eps = b + plane * 3;
    for (int m = 0; m < 3; ++m) r->S.w[m] = b + plane * (4 + m);
    r->S.F = b + plane * 7;
    r->S.E = b + plane * 8;
    for (int m = 0; m < 3; ++m) r->S.P[m] = b + plane * (9 + m);
    r->S.qb[0] = r->S.eps;
    for (int m = 0; m < 3; ++m) r->S.qb[1 + m] = r->S.w[m];
    r->S.qb[4] = r->S.P[0];
  }
  CKR(dev_alloc(r->al, (void**)&r->ds, sizeof(DevScalars)));
  CKR(cudaMemset(r->ds, 0, sizeof(DevScalars)));
  // partials: 3 per force block of every level, and one per 256 active cells of a
  // level for the luminosity normalisation (the two uses never overlap in time)
  int np = 0;
  for (int l = 0; l < n_levels; ++l) np += force_partials_per_level(r->L[l].v);
  r->n_partials = np;
  size_t pelems = std::max(3 * (size_t)np, (na_max + 255) / 256);
  CKR(dev_alloc(r->al, (void**)&r->partials, pelems * sizeof(double)));
  CKR(dev_alloc(r->al, (void**)&r->ring, kRingStride * (size_t)r->ring_cap * sizeof(double)));
  CKR(dev_alloc(r->al, (void**)&r->ring_pos, sizeof(long long)));
  CKR(cudaMemset(r->ring_pos, 0, sizeof(long long)));
  CKR(dev_alloc(r->al, (void**)&r->wsum, sizeof(double)));
  CKR(dev_alloc(r->al, (void**)&r->stage, r->nc_max * sizeof(double)));
#undef CKR
  *out = r;
  return DF_OK;
}

int check_params(const df_params* p) {
  if (!p) return fail(DF_EINVAL, "null params");
  if (!(p->gamma > 1.0) || !(p->rho0 > 0.0) || !(p->cs > 0.0) || p->chi < 0.0 ||
      !(p->cfl > 0.0) || p->band < 1 || p->mach < 0.0)
    return fail(DF_EINVAL, "invalid physical parameters");
  if (p->chi > 0.0 && !(p->cfl_diff > 0.0)) return fail(DF_EINVAL, "cfl_diff must be > 0");
  if (!(p->av_c2 >= 0.0) || !std::isfinite(p->av_c2))
    return fail(DF_EINVAL, "av_c2 must be finite and >= 0");
  for (int k = 0; k < 6; ++k)
    if (p->bc[k] < 0 || p->bc[k] > 3) return fail(DF_EINVAL, "bad boundary type");
  return DF_OK;
}

// parameters, uniform background state, static fields; returns kernels launched
long long run_set_params(Run* r, const df_params* p, cudaStream_t st, int* rc) {
  *rc = DF_OK;
  r->prm = *p;
  Phys& P = r->P;
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
  P.av_c2 = p->av_c2;
  for (int k = 0; k < 6; ++k) P.bc[k] = p->bc[k];
  const int mir = mirror_mask(r->lo, p);
  P.mult = 1.0;
  for (int d = 0; d < 3; ++d)
    if (mir >> d & 1) P.mult *= 2.0;
  long long n = 0;
  for (int l = 0; l < r->nl; ++l) r->L[l].v.mir = mir;
  for (int l = 0; l < r->nl; ++l) {
    LevelView& v = r->L[l].v;
    if (r->prec == DF_FP64) {
      n += launch_init_uniform<double>(v, P, st);
      n += launch_static_fields<double>(v, P, p->lum_sigma, r->wsum, r->partials, st);
      if (p->lum_sigma > 0.0) n += launch_normalise_lum<double>(v, r->wsum, P.mult, st);
    } else {
      n += launch_init_uniform<float>(v, P, st);
      n += launch_static_fields<float>(v, P, p->lum_sigma, r->wsum, r->partials, st);
      if (p->lum_sigma > 0.0) n += launch_normalise_lum<float>(v, r->wsum, P.mult, st);
    }
    if (cudaMemsetAsync(r->L[l].acc, 0, r->L[l].acc_elems * sizeof(double), st) != cudaSuccess)
      *rc = fail(DF_ECUDA, "memset");
    n += launch_force_weights(v, P, st);
  }
  DevScalars h;
  memset(&h, 0, sizeof h);  // per-axis maxima start at +0.0 (bit pattern 0)
  if (cudaMemcpyAsync(r->ds, &h, sizeof h, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(r->ring_pos, 0, sizeof(long long), st) != cudaSuccess)
    *rc = fail(DF_ECUDA, "scalar reset");
  r->have_params = true;
  r->stepped = false;
  return n;
}

// ------------------------------------------------------------------------ plans

struct LaunchDesc {
  int op, d, kind;
  size_t item0, start0;
  int nitems;
  unsigned nchunks;
};

struct Plan {
  int prec = 0;
  size_t item_size = 0;
  std::vector<LaunchDesc> launches;
  std::vector<unsigned char> items;  // host copy, item_size bytes each
  std::vector<unsigned> starts;
  std::vector<DtFinal> fins;
  void* d_items = nullptr;
  unsigned* d_starts = nullptr;
  DtFinal* d_fins = nullptr;
  size_t cap_items = 0, cap_starts = 0, cap_fins = 0;
  cudaGraphExec_t gexec = nullptr;
  long long kernels = 0;
  bool valid = false;
  Allocator al;  // the owner's
};

void plan_free(Plan& p) {
  if (p.gexec) cudaGraphExecDestroy(p.gexec);
  dev_free(p.al, p.d_items);
  dev_free(p.al, p.d_starts);
  dev_free(p.al, p.d_fins);
  const Allocator al = p.al;
  p = Plan();
  p.al = al;
}

void plan_invalidate(Plan& p) {
  if (p.gexec) {
    cudaGraphExecDestroy(p.gexec);
    p.gexec = nullptr;
  }
  p.valid = false;
}

int kind_of(int op) {
  switch (op) {
    case OP_BC: return K_BC;
    case OP_SOURCE: return K_SOURCE;
    case OP_COMPRESS: return K_COMPRESS;
    case OP_DIFFUSE: return K_DIFFUSE;
    case OP_FRONTIER_DIFF: return K_FRONTIER_DIFF;
    case OP_TPREP: return K_TPREP;
    case OP_TFLUX: return K_TFLUX;
    case OP_TFRONTIER: return K_TFRONTIER;
    case OP_TMOM: return K_TMOM;
    case OP_TUPDATE: return K_TUPDATE;
    case OP_VREC: return K_VREC_SOURCE;
    case OP_COMMUP: return K_COMMUP;
    case OP_COMMMEAN: return K_COMMMEAN;
    case OP_DT_LEVEL: case OP_DT_FINAL: return K_DT;
    case OP_FORCE_LEVEL: case OP_FORCE_FINAL: return K_FORCE;
    case OP_SWEEP: return K_SWEEP;
    case OP_VISC_Q: case OP_VISC_V: return K_VISC;
    default: return K_OTHER;
  }
}

void fill_fin(const Run& r, DtFinal& fin) {
  double pr = 1.0;
  fin.search = 0;
  fin.pad = 0;
  for (int l = 0; l < 16; ++l) {
    fin.prod[l] = 1.0;
    fin.cost[l] = 0.0;
    fin.diff_lim[l] = INFINITY;
    for (int d = 0; d < 3; ++d) fin.cfl_dx[l][d] = 0.0;
    for (int q = 0; q < 12; ++q) fin.kfac[l][q] = 0.0;
  }
  for (int l = 0; l < r.nl; ++l) {
    if (l > 0) pr *= r.xi[l - 1];
    fin.prod[l] = pr;
    const LevelView& v = r.L[l].v;
    if (r.P.chi > 0.0) {
      double sinv = 0.0;
      for (int d = 0; d < 3; ++d) sinv += 1.0 / (v.dx[d] * v.dx[d]);
      fin.diff_lim[l] = r.P.cfl_diff / (2.0 * r.P.chi * sinv);
    }
    for (int d = 0; d < 3; ++d) fin.cfl_dx[l][d] = r.P.hydro_on ? r.P.cfl * v.dx[d] : 0.0;
    for (int d = 0; d < 3; ++d) {
      fin.kfac[l][K_ADT + d] = v.area[d];
      fin.kfac[l][K_DTDX + d] = v.inv_dx[d];
      fin.kfac[l][K_DIFF + d] = -r.P.chi * v.dcoef[d];
      fin.kfac[l][K_F0 + d] = r.P.rho0 * r.P.V[d] * v.area[d];
    }
    fin.cost[l] = (double)v.n[0] * v.n[1] * v.n[2];
  }
  fin.search = r.prm.xi_mode == 1 && r.nl > 1;
}

// tile shape (index into kTileShapes) of each stencil op and sweep direction
struct TileTable {
  int t[OP_COUNT][3];
  TileTable() {
    for (int o = 0; o < OP_COUNT; ++o)
      for (int d = 0; d < 3; ++d) t[o][d] = 0;
  }
};

// Transport of one level step: DF_TRANSPORT_FUSED or DF_TRANSPORT_SEPARATE as set.
// DF_TRANSPORT_AUTO picks separate kernels for FP64, whose kernels are bound by the
// FP64 pipe, which the halo arithmetic the sweeps repeat would load further.  For
// the FP32 state it picks fused sweeps in pools, whose merged launches give the
// sweeps blocks enough (and a run must get the same bits whatever it shares its
// pool with), and for a context's levels of at least kFusedMinCells active cells.
// A fused sweep's blocks march through whole columns, so one small box leaves the
// GPU short of blocks: on GB300 the separate kernels win for one run of 3 x 64^3
// levels, the sweeps from 3 x 96^3, and the sweeps win for pools of small runs.
constexpr long long kFusedMinCells = 512 * 1024;

bool sweeps_fused(int mode, int prec, const LevelView& v, bool pool) {
  if (mode != DF_TRANSPORT_AUTO) return mode == DF_TRANSPORT_FUSED;
  return prec == DF_FP32_STATE &&
         (pool || (long long)v.n[0] * v.n[1] * v.n[2] >= kFusedMinCells);
}

template <class T>
struct Builder {
  struct Entry {
    int op, d;
    Item<T> it;
  };
  std::vector<std::vector<Entry>> per_run;
  int full_boxes = 0;
  const DtFinal* d_fins = nullptr;
  TileTable tiles;
  int transport = DF_TRANSPORT_AUTO;  // per level: fused sweeps or separate kernels
  bool pool = false;                  // the plan steps a pool (else a context)
  mutable unsigned br = 0;  // second sub-cycles enclosing the items being added
  mutable int sub_of[DF_MAX_LEVELS] = {};  // sub-cycle of each level being added

  Item<T> base(const Run& r, int l) const {
    Item<T> it;
    memset(&it, 0, sizeof it);
    it.L = r.L[l].v;
    // the active box: the enumeration of the time-step and force reductions (box ops
    // set their own)
    for (int d = 0; d < 3; ++d) {
      it.b.lo[d] = it.L.G;
      it.b.hi[d] = it.L.G + it.L.n[d];
    }
    it.b.set_divisors();
    it.S = r.S;
    using C = Arith<T>;
    it.bg = make_bg<C>(r.P);
    it.g = make_geo<C>(it.L);
    it.dt = sizeof(T) == 8 ? (const void*)&r.ds->dtd[l] : (const void*)&r.ds->dtf[l];
    it.kc = sizeof(T) == 8 ? (const void*)&r.ds->kd[l][0] : (const void*)&r.ds->kf[l][0];
    it.ds = r.ds;
    it.gm1 = to_arith<C>(r.P.gamma - 1.0);
    it.lum = to_arith<C>(r.P.L);
    it.av = to_arith<C>(r.P.av_c2);
    it.gg = r.P.gamma * (r.P.gamma - 1.0);
    it.gga = to_arith<C>(it.gg);
    it.rho0d = r.P.rho0;
    it.e0d = r.P.e0;
    for (int d = 0; d < 3; ++d) it.V[d] = r.P.V[d];
    it.dt_fixed = r.P.dt_fixed;
    it.level = l;
    it.sub = sub_of[l];
    it.band = r.P.band;
    int fl = 0;
    if (r.P.hydro_on) fl |= FL_HYDRO | FL_SS3 | FL_WRITE_PI;
    if (r.P.L != 0.0) fl |= FL_LUM;
    if (r.P.chi > 0.0) fl |= FL_EPS;
    if (r.P.diff_face_rho) fl |= FL_DFR;
    it.flags = fl;
    return it;
  }

  // planes per chunk of a fused sweep's marching axis, at least 8 (16 when marching
  // along the sweep, whose chunks start 3 planes early and finish 2 planes late).
  // A context's sweep launches one block per (column, chunk): as many chunks as
  // leave every block resident at once (one wave: the SMs times the blocks of that
  // kernel an SM holds, when that is at least two), since each chunk repeats the
  // planes of its halo.  A pool's persistent blocks take chunks in turn: about 600
  // chunks balance them.
  int sweep_chunk(const Box& b, int d) const {
    const int ra = sweep_row_axis(d), mu = sweep_march_axis(d), ow = sweep_own_x(d);
    const int ncols = ((b.hi[0] - b.lo[0] + ow - 1) / ow) *
                      ((b.hi[ra] - b.lo[ra] + kSweepRows - 1) / kSweepRows);
    const int nm = b.hi[mu] - b.lo[mu];
    const int slots = pool ? 600 : sweep_slots((int)sizeof(T), d);
    const int chunks = std::max(1, slots / std::max(1, ncols));
    const int zc = (nm + chunks - 1) / chunks;
    return std::min(nm, std::max(zc, d == 0 ? 8 : 16));
  }

  // margin boxes (active cells +- margin) unless verifying with whole arrays or the
  // artificial viscosity is on (its viscous pressures one cell below a box edge are
  // not formed by a margin box, and the reach behind the margins was measured
  // without it): then every operator sweeps the whole padded array
  // On level 0 the upper boundary face G + n of v_d is the solver's and keeps its
  // value from one level step to the next, as the lower face G does, so the box
  // reaches one element further up: the margin covers the reach of one level step
  // above that face too.
  Box box(const LevelView& v, int margin, bool whole = false, int up = 0) const {
    Box b;
    b.tile = 0;
    b.zc = 0;
    int M = (full_boxes || whole) ? v.G : margin;
    for (int d = 0; d < 3; ++d) {
      b.lo[d] = std::max(0, v.G - M);
      b.hi[d] = std::min(v.s[d], v.G + v.n[d] + M + up);
    }
    b.set_divisors();
    return b;
  }

  void add(std::vector<Entry>& out, int op, int d, Item<T> it) const {
    it.b.tile = is_box_op(op) ? tiles.t[op][d] : 0;
    it.b.zc = op == OP_SWEEP ? sweep_chunk(it.b, d) : 0;
    it.br = br;
    it.count = op_count(op, d, it.L, it.F, it.b);
    out.push_back({op, d, it});
  }

  // reflect fill of the mirror sides only (type -1: the upper side is left alone)
  void mirror_fill(const Item<T>& it, std::vector<Entry>& out) const {
    for (int d = 0; d < 3; ++d)
      if (it.L.mir >> d & 1) {
        Item<T> bc = it;
        bc.bc_lo = DF_BC_REFLECT;
        bc.bc_hi = -1;
        add(out, OP_BC, d, bc);
      }
  }

  void level_step(const Run& r, int l, int m_out, std::vector<Entry>& out) const {
    Item<T> it = base(r, l);
    it.b = box(it.L, m_out + kReach, r.P.av_c2 > 0.0, l == 0 ? 1 : 0);
    const Phys& P = r.P;
    // The two sub-cycles of a finest level follow each other with nothing in between
    // that changes it (no boundary fill, CommUp or CommMean; no mirror fill where it
    // has no mirror plane; both always run without the Eq. 55-56 search): the first
    // one's velocity recovery also applies the second one's first kick.
    const bool paired = P.hydro_on && l > 0 && l + 1 == r.nl && r.xi[l - 1] == 2 &&
                        r.prm.xi_mode != 1 && it.L.mir == 0;
    const bool kick_done = paired && sub_of[l] == 1;
    const int vrec_d = paired && sub_of[l] == 0 ? 1 : 0;
    if (l == 0)
      for (int d = 0; d < 3; ++d) {
        Item<T> bc = it;
        bc.bc_lo = P.bc[2 * d];
        bc.bc_hi = P.bc[2 * d + 1];
        add(out, OP_BC, d, bc);
      }
    else
      mirror_fill(it, out);  // CommUp filled the rest of the ghosts
    if (P.hydro_on && !kick_done) add(out, OP_SOURCE, 0, it);
    if (P.hydro_on && P.av_c2 > 0.0) {
      add(out, OP_VISC_Q, 0, it);
      add(out, OP_VISC_V, 0, it);
    }
    if (P.hydro_on || P.L != 0.0 || P.chi > 0.0) add(out, OP_COMPRESS, 0, it);
    const bool fused_tr =
        sweeps_fused(transport, sizeof(T) == 8 ? DF_FP64 : DF_FP32_STATE, it.L, pool);
    // before the separate transport kernels the diffusion also forms the x sweep's
    // e/rho (in Scratch::w[0]), in place of that sweep's preparation kernel
    const bool eps_x = P.chi > 0.0 && P.hydro_on && !fused_tr;
    if (P.chi > 0.0) {
      if (it.L.is_child) add(out, OP_FRONTIER_DIFF, 0, it);
      add(out, OP_DIFFUSE, eps_x ? 1 : 0, it);
    }
    if (P.hydro_on && fused_tr) {
      for (int d = 0; d < 3; ++d) {
        add(out, OP_SWEEP, d, it);
      }
      Item<T> vr = it;
      vr.flags |= FL_FUSED;
      add(out, OP_VREC, vrec_d, vr);
    } else if (P.hydro_on) {
      // At the x sweep the staggered momenta were just formed from v and rho (the
      // kick, or the viscosity stage after it, wrote them; nothing since has changed
      // v or rho), so Pi/rho_face - V is the velocity deviation itself: that sweep's
      // momentum fluxes read v, and its preparation forms e/rho only.  The y and z
      // sweeps divide the updated momenta.
      for (int d = 0; d < 3; ++d) {
        Item<T> tp = it, tm = it, tf = it;
        if (d == 0) {
          tp.flags |= FL_EPS_ONLY;
          for (int m = 0; m < 3; ++m) tm.S.w[m] = it.L.q[F_VX + m];
          if (eps_x) tf.S.eps = it.S.w[0];
        }
        if (d > 0 || !eps_x) add(out, OP_TPREP, 0, tp);
        add(out, OP_TFLUX, d, tf);
        add(out, OP_TMOM, d, tm);
        add(out, OP_TUPDATE, d, it);
      }
      add(out, OP_VREC, vrec_d, it);
    }
  }

  void advance(const Run& r, int l, int m_out, std::vector<Entry>& out) const {
    if (l + 1 < r.nl) {
      int xi = r.xi[l];
      for (int s = 0; s < xi; ++s) {
        // the second sub-cycle (and all it encloses) is dropped on the device when
        // the Eq. 55-56 search picks xi_l = 1; the first keeps the margin of two.
        // Each sub-cycle writes its own part of the child's CommFlux record, so the
        // record needs no clearing: the parent sums the parts of the sub-cycles run.
        const unsigned saved = br;
        if (s == 1) br |= 1u << l;
        sub_of[l + 1] = s;
        advance(r, l + 1, (xi - 1 - s) * kReach, out);
        br = saved;
      }
      sub_of[l + 1] = 0;
    }
    level_step(r, l, m_out, out);
    if (l + 1 < r.nl) {
      Item<T> it = base(r, l);
      mirror_fill(it, out);  // the CommUp stencil reaches across a mirror plane
      it.F = r.L[l + 1].v;
      add(out, OP_COMMUP, 0, it);
      add(out, OP_COMMMEAN, 0, it);
    }
  }

  Item<T> force_level_item(const Run& r, int l) const {
    Item<T> f = base(r, l);
    int off = 0;
    for (int m = 0; m < l; ++m) off += force_partials_per_level(r.L[m].v);
    f.partials = r.partials + 3 * off;
    return f;
  }

  Item<T> force_final_item(const Run& r, bool ring) const {
    Item<T> ff = base(r, 0);
    ff.partials = r.partials;
    ff.npart = r.n_partials;
    if (ring) {
      ff.ring = r.ring;
      ff.ring_pos = r.ring_pos;
      ff.ring_cap = r.ring_cap;
    }
    return ff;
  }

  void coarse_step(const Run& r, int ri, std::vector<Entry>& out) const {
    for (int l = 0; l < r.nl; ++l) add(out, OP_DT_LEVEL, 0, base(r, l));
    Item<T> fin = base(r, 0);
    fin.level = r.nl;  // the finalisation covers all levels
    fin.fin = d_fins + ri;
    add(out, OP_DT_FINAL, 0, fin);
    advance(r, 0, 0, out);
    for (int l = 0; l < r.nl; ++l) add(out, OP_FORCE_LEVEL, 0, force_level_item(r, l));
    add(out, OP_FORCE_FINAL, 0, force_final_item(r, true));
    add(out, OP_TIME, 0, base(r, 0));
  }

  // greedy merge: repeatedly launch the op kind that heads the most runs' lists,
  // taking it from every run whose next op it is (each run keeps its own order)
  void merge(Plan& plan) const {
    size_t nr = per_run.size();
    std::vector<size_t> pos(nr, 0);
    plan.item_size = sizeof(Item<T>);
    plan.items.clear();
    plan.starts.clear();
    plan.launches.clear();
    for (;;) {
      std::map<std::pair<int, int>, int> cnt;
      for (size_t r = 0; r < nr; ++r)
        if (pos[r] < per_run[r].size()) cnt[{per_run[r][pos[r]].op, per_run[r][pos[r]].d}]++;
      if (cnt.empty()) break;
      std::pair<int, int> best = cnt.begin()->first;
      int bc = -1;
      for (auto& kv : cnt)
        if (kv.second > bc) {
          bc = kv.second;
          best = kv.first;
        }
      LaunchDesc L;
      L.op = best.first;
      L.d = best.second;
      L.kind = kind_of(L.op);
      L.item0 = plan.items.size() / plan.item_size;
      L.start0 = plan.starts.size();
      L.nitems = 0;
      unsigned chunks = 0;
      unsigned ce = (unsigned)op_chunk_elems(L.op, (int)sizeof(T));
      for (size_t r = 0; r < nr; ++r) {
        if (pos[r] >= per_run[r].size()) continue;
        const Entry& e = per_run[r][pos[r]];
        if (e.op != best.first || e.d != best.second) continue;
        ++pos[r];
        unsigned nch = (e.it.count + ce - 1) / ce;
        if (nch == 0) continue;
        const unsigned char* p = reinterpret_cast<const unsigned char*>(&e.it);
        plan.items.insert(plan.items.end(), p, p + sizeof(Item<T>));
        plan.starts.push_back(chunks);
        chunks += nch;
        ++L.nitems;
      }
      L.nchunks = chunks;
      if (L.nitems) plan.launches.push_back(L);
    }
  }
};

int grow(const Allocator& a, void** p, size_t* cap, size_t need) {
  if (need <= *cap) return DF_OK;
  dev_free(a, *p);
  *p = nullptr;
  *cap = 0;
  size_t c = std::max(need, (size_t)4096);
  CK(dev_alloc(a, p, c));
  *cap = c;
  return DF_OK;
}

int plan_upload(Plan& plan) {
  int rc = grow(plan.al, &plan.d_items, &plan.cap_items, plan.items.size());
  if (rc) return rc;
  rc = grow(plan.al, (void**)&plan.d_starts, &plan.cap_starts, plan.starts.size() * sizeof(unsigned));
  if (rc) return rc;
  if (!plan.items.empty())
    CK(cudaMemcpy(plan.d_items, plan.items.data(), plan.items.size(), cudaMemcpyHostToDevice));
  if (!plan.starts.empty())
    CK(cudaMemcpy(plan.d_starts, plan.starts.data(), plan.starts.size() * sizeof(unsigned),
                  cudaMemcpyHostToDevice));
  return DF_OK;
}

template <class T>
int plan_build(Plan& plan, const std::vector<Run*>& runs, int full_boxes,
               const TileTable& tiles, int transport, bool pool) {
  plan_invalidate(plan);
  plan.prec = sizeof(T) == 8 ? DF_FP64 : DF_FP32_STATE;
  size_t nr = runs.size();
  plan.fins.resize(std::max<size_t>(nr, 1));
  for (size_t r = 0; r < nr; ++r) fill_fin(*runs[r], plan.fins[r]);
  int rc = grow(plan.al, (void**)&plan.d_fins, &plan.cap_fins, plan.fins.size() * sizeof(DtFinal));
  if (rc) return rc;
  CK(cudaMemcpy(plan.d_fins, plan.fins.data(), plan.fins.size() * sizeof(DtFinal),
                cudaMemcpyHostToDevice));
  Builder<T> B;
  B.full_boxes = full_boxes;
  B.d_fins = plan.d_fins;
  B.tiles = tiles;
  B.transport = transport;
  B.pool = pool;
  B.per_run.resize(nr);
  for (size_t r = 0; r < nr; ++r) B.coarse_step(*runs[r], (int)r, B.per_run[r]);
  B.merge(plan);
  rc = plan_upload(plan);
  if (rc) return rc;
  plan.valid = true;
  return DF_OK;
}

// a plan of explicitly listed ops of one run (inter-level operators on demand, the
// force of the current state, the time-step reduction alone)
template <class T>
int plan_build_ops(Plan& plan, Run* r, const std::vector<std::pair<int, int>>& ops) {
  plan_invalidate(plan);
  plan.prec = sizeof(T) == 8 ? DF_FP64 : DF_FP32_STATE;
  plan.fins.resize(1);
  fill_fin(*r, plan.fins[0]);
  int rc = grow(plan.al, (void**)&plan.d_fins, &plan.cap_fins, sizeof(DtFinal));
  if (rc) return rc;
  CK(cudaMemcpy(plan.d_fins, plan.fins.data(), sizeof(DtFinal), cudaMemcpyHostToDevice));
  Builder<T> B;
  B.d_fins = plan.d_fins;
  B.per_run.resize(1);
  auto& v = B.per_run[0];
  for (auto& ol : ops) {
    int op = ol.first, l = ol.second;
    Item<T> it = B.base(*r, l);
    // box ops over the whole array; the reductions keep base()'s active box
    if (op != OP_DT_LEVEL && op != OP_FORCE_LEVEL) it.b = B.box(it.L, it.L.G);
    switch (op) {
      case OP_COMMUP:
        B.mirror_fill(it, v);  // as in the coarse step: the stencil reaches across a plane
        it.F = r->L[l + 1].v;
        B.add(v, op, 0, it);
        break;
      case OP_COMMMEAN:
        it.F = r->L[l + 1].v;
        B.add(v, op, 0, it);
        break;
      case OP_BC:
        for (int d = 0; d < 3; ++d) {
          Item<T> bc = it;
          bc.bc_lo = r->P.bc[2 * d];
          bc.bc_hi = r->P.bc[2 * d + 1];
          B.add(v, OP_BC, d, bc);
        }
        break;
      case OP_FORCE_LEVEL:
        B.add(v, op, 0, B.force_level_item(*r, l));
        break;
      case OP_FORCE_FINAL:
        B.add(v, op, 0, B.force_final_item(*r, false));
        break;
      case OP_DT_FINAL:
        it.level = r->nl;
        it.fin = plan.d_fins;
        B.add(v, op, 0, it);
        break;
      default:
        B.add(v, op, 0, it);
    }
  }
  B.merge(plan);
  rc = plan_upload(plan);
  if (rc) return rc;
  plan.valid = true;
  return DF_OK;
}

// ---------------------------------------------------------------- execution

struct Exec {
  cudaStream_t st = nullptr;
  int sm_count = 148;
  int bps[OP_COUNT];  // persistent blocks per SM of each op (autotuned for pools)
  bool timing = false;
  struct EvPair {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<EvPair> evpool;
  size_t ev_used = 0;
  double k_ms[K_NKINDS] = {};
  long long k_n[K_NKINDS] = {};
  long long launches = 0;
  bool single_fast = true;  // contexts: one-item launches pass the item by value
  Exec() {
    for (int o = 0; o < OP_COUNT; ++o) bps[o] = 8;
  }
};

bool exec_init(Exec& x, int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms)
    x.sm_count = sms;
  return true;
}

void exec_free(Exec& x) {
  for (auto& p : x.evpool) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  x.evpool.clear();
}

// Fold the recorded event pairs into the per-kind totals (synchronises).
void harvest_timing(Exec& x) {
  if (!x.ev_used) return;
  cudaStreamSynchronize(x.st);
  for (size_t i = 0; i < x.ev_used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, x.evpool[i].a, x.evpool[i].b);
    x.k_ms[x.evpool[i].kind] += ms;
    x.k_n[x.evpool[i].kind] += 1;
  }
  x.ev_used = 0;
}

template <class T>
long long plan_run(const Plan& plan, Exec& x, bool events) {
  long long n = 0;
  const unsigned char* items = (const unsigned char*)plan.d_items;
  for (const LaunchDesc& L : plan.launches) {
    unsigned grid = (unsigned)x.sm_count * (unsigned)x.bps[L.op];
    const Item<T>* it = (const Item<T>*)(items + L.item0 * plan.item_size);
    const unsigned* st = plan.d_starts + L.start0;
    const Item<T>* hi = (L.nitems == 1 && x.single_fast)
                            ? (const Item<T>*)(plan.items.data() + L.item0 * plan.item_size)
                            : nullptr;
    if (events) {
      if (x.ev_used == x.evpool.size()) {
        Exec::EvPair p;
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        x.evpool.push_back(p);
      }
      Exec::EvPair& p = x.evpool[x.ev_used++];
      p.kind = L.kind;
      cudaEventRecord(p.a, x.st);
      n += launch_batch<T>(L.op, L.d, it, st, L.nitems, L.nchunks, grid, x.st, hi);
      cudaEventRecord(p.b, x.st);
    } else {
      n += launch_batch<T>(L.op, L.d, it, st, L.nitems, L.nchunks, grid, x.st, hi);
    }
  }
  return n;
}

// nsteps coarse steps of every run of the plan: graph replay, or direct launches
// bracketed by events in timing mode
template <class T>
int plan_step(Plan& plan, Exec& x, int nsteps) {
  if (x.timing) {
    for (int s = 0; s < nsteps; ++s) x.launches += plan_run<T>(plan, x, true);
    CK(cudaGetLastError());
    return DF_OK;
  }
  if (!plan.gexec) {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(x.st, cudaStreamCaptureModeThreadLocal));
    long long n = plan_run<T>(plan, x, false);
    cudaError_t e = cudaStreamEndCapture(x.st, &g);
    if (e != cudaSuccess) return fail(DF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&plan.gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(DF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    plan.kernels = n;
  }
  for (int s = 0; s < nsteps; ++s) {
    CK(cudaGraphLaunch(plan.gexec, x.st));
    x.launches += plan.kernels;
  }
  return DF_OK;
}

// run a list of ops of one run now, without a graph, and wait for it
int run_ops_now(Run* r, Exec& x, const std::vector<std::pair<int, int>>& ops) {
  Plan p;
  p.al = r->al;
  int rc = r->prec == DF_FP64 ? plan_build_ops<double>(p, r, ops) : plan_build_ops<float>(p, r, ops);
  if (!rc) {
    x.launches += r->prec == DF_FP64 ? plan_run<double>(p, x, false) : plan_run<float>(p, x, false);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(x.st);
    if (e != cudaSuccess) rc = fail(DF_ECUDA, "ops: %s", cudaGetErrorString(e));
  }
  plan_free(p);
  return rc;
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

// background value of a field (the stored state is the deviation from it)
double field_bg(const Run* r, int field) {
  return field == 0 ? r->P.rho0 : field == 1 ? r->P.e0 : r->P.V[field - 2];
}

template <class T>
int run_io(Run* r, cudaStream_t st, int level, int field, double* out, const double* in, int full,
           bool raw, long long* launches) {
  if (level < 0 || level >= r->nl || field < 0 || field > 4)
    return fail(DF_EINVAL, "level %d / field %d out of range", level, field);
  LevelView& v = r->L[level].v;
  size_t n = full ? (size_t)v.nc : (size_t)v.n[0] * v.n[1] * v.n[2];
  double bgv = raw ? 0.0 : field_bg(r, field);
  if (in) {
    CK(cudaMemcpyAsync(r->stage, in, n * sizeof(double), cudaMemcpyHostToDevice, st));
    *launches += launch_unpack_active<T>(v, field, r->stage, full, bgv, st);
  } else {
    *launches += launch_pack_active<T>(v, field, r->stage, full, bgv, st);
    CK(cudaMemcpyAsync(out, r->stage, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return DF_OK;
}

int io(Run* r, cudaStream_t st, int level, int field, double* out, const double* in, int full,
       bool raw, long long* launches) {
  return r->prec == DF_FP64 ? run_io<double>(r, st, level, field, out, in, full, raw, launches)
                            : run_io<float>(r, st, level, field, out, in, full, raw, launches);
}

}  // namespace

// --------------------------------------------------------------------- contexts

struct df_ctx {
  int device = 0;
  cudaStream_t user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  Run* run = nullptr;
  Plan plan;
  Exec x;
  int full_boxes = 0;
  TileTable tiles;
  int transport = DF_TRANSPORT_AUTO;
};

struct df_pool {
  int device = 0, prec = 0;
  size_t budget = 0, used = 0;
  cudaStream_t user = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<Run*> slots;
  Plan plan;
  Exec x;
  TileTable tiles;
  int transport = DF_TRANSPORT_AUTO;
};

namespace {

template <class C>
void enter(C* c) {
  cudaEventRecord(c->ev_in, c->user);
  cudaStreamWaitEvent(c->x.st, c->ev_in, 0);
}
template <class C>
void leave(C* c) {
  cudaEventRecord(c->ev_out, c->x.st);
  cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

int check_ctx(df_ctx* c, bool need_params = true) {
  if (!c || !c->run) return fail(DF_EINVAL, "null context");
  if (need_params && !c->run->have_params) return fail(DF_EINVAL, "df_set_params not called");
  return DF_OK;
}

int sync_health(cudaStream_t st, Run* r) {
  CK(cudaStreamSynchronize(st));
  int bad = 0;
  CK(cudaMemcpy(&bad, &r->ds->unhealthy, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) return fail(DF_EUNHEALTHY, "NaN, rho <= 0 or e <= 0 found in the state");
  return DF_OK;
}

int build_plan(Plan& p, const std::vector<Run*>& runs, int prec, int full_boxes,
               const TileTable& tiles, int transport, bool pool) {
  return prec == DF_FP64 ? plan_build<double>(p, runs, full_boxes, tiles, transport, pool)
                         : plan_build<float>(p, runs, full_boxes, tiles, transport, pool);
}

// state of the runs that tuning steps disturb (fields, scalars, force-ring cursor)
struct Snapshot {
  std::vector<std::vector<char>> fields, acc, ring;
  std::vector<DevScalars> ds;
  std::vector<long long> pos;
};

int snapshot(const std::vector<Run*>& runs, Snapshot& sn) {
  sn.fields.assign(runs.size(), {});
  sn.acc.assign(runs.size(), {});
  sn.ring.assign(runs.size(), {});
  sn.ds.resize(runs.size());
  sn.pos.resize(runs.size());
  for (size_t i = 0; i < runs.size(); ++i) {
    Run* r = runs[i];
    // level l at offset l * (largest level's size): levels differ with a ground level
    size_t pmax = plane_bytes(r->nc_max, r->esz), amax = 0;
    for (int l = 0; l < r->nl; ++l) amax = std::max(amax, r->L[l].acc_elems * sizeof(double));
    sn.fields[i].resize(pmax * 5 * r->nl);
    sn.acc[i].resize(amax * r->nl);
    for (int l = 0; l < r->nl; ++l) {
      size_t plane = plane_bytes((size_t)r->L[l].v.nc, r->esz);
      size_t ab = r->L[l].acc_elems * sizeof(double);
      CK(cudaMemcpy(sn.fields[i].data() + pmax * 5 * l, r->L[l].mem, plane * 5,
                    cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(sn.acc[i].data() + amax * l, r->L[l].acc, ab, cudaMemcpyDeviceToHost));
    }
    sn.ring[i].resize(kRingStride * (size_t)r->ring_cap * sizeof(double));
    CK(cudaMemcpy(sn.ring[i].data(), r->ring, sn.ring[i].size(), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&sn.ds[i], r->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&sn.pos[i], r->ring_pos, sizeof(long long), cudaMemcpyDeviceToHost));
  }
  return DF_OK;
}

int restore(const std::vector<Run*>& runs, const Snapshot& sn) {
  for (size_t i = 0; i < runs.size(); ++i) {
    Run* r = runs[i];
    size_t pmax = plane_bytes(r->nc_max, r->esz), amax = 0;
    for (int l = 0; l < r->nl; ++l) amax = std::max(amax, r->L[l].acc_elems * sizeof(double));
    for (int l = 0; l < r->nl; ++l) {
      size_t plane = plane_bytes((size_t)r->L[l].v.nc, r->esz);
      size_t ab = r->L[l].acc_elems * sizeof(double);
      CK(cudaMemcpy(r->L[l].mem, sn.fields[i].data() + pmax * 5 * l, plane * 5,
                    cudaMemcpyHostToDevice));
      CK(cudaMemcpy(r->L[l].acc, sn.acc[i].data() + amax * l, ab, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(r->ring, sn.ring[i].data(), sn.ring[i].size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(r->ds, &sn.ds[i], sizeof(DevScalars), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(r->ring_pos, &sn.pos[i], sizeof(long long), cudaMemcpyHostToDevice));
  }
  return DF_OK;
}

// Device time of every launch of one coarse step of `p`, summed per (op, direction):
// two coarse steps run back to back and the second is timed.  bps > 0 overrides
// the persistent blocks per SM of every launch.
int time_plan(const Plan& p, Exec& x, int prec, int bps, bool single_fast,
              double per[OP_COUNT][3]) {
  for (int o = 0; o < OP_COUNT; ++o)
    for (int d = 0; d < 3; ++d) per[o][d] = 0.0;
  std::vector<cudaEvent_t> ev(2 * p.launches.size());
  for (auto& e : ev) CK(cudaEventCreate(&e));
  const unsigned char* items = (const unsigned char*)p.d_items;
  for (int rep = 0; rep < 2; ++rep)
    for (size_t i = 0; i < p.launches.size(); ++i) {
      const LaunchDesc& L = p.launches[i];
      unsigned grid = (unsigned)x.sm_count * (unsigned)(bps > 0 ? bps : x.bps[L.op]);
      const void* hi = (L.nitems == 1 && single_fast)
                           ? (const void*)(p.items.data() + L.item0 * p.item_size)
                           : nullptr;
      if (rep == 1) cudaEventRecord(ev[2 * i], x.st);
      if (prec == DF_FP64)
        launch_batch<double>(L.op, L.d, (const Item<double>*)(items + L.item0 * p.item_size),
                             p.d_starts + L.start0, L.nitems, L.nchunks, grid, x.st,
                             (const Item<double>*)hi);
      else
        launch_batch<float>(L.op, L.d, (const Item<float>*)(items + L.item0 * p.item_size),
                            p.d_starts + L.start0, L.nitems, L.nchunks, grid, x.st,
                            (const Item<float>*)hi);
      if (rep == 1) cudaEventRecord(ev[2 * i + 1], x.st);
    }
  cudaError_t e = cudaStreamSynchronize(x.st);
  for (size_t i = 0; e == cudaSuccess && i < p.launches.size(); ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
    per[p.launches[i].op][p.launches[i].d] += ms;
  }
  for (auto& v : ev) cudaEventDestroy(v);
  if (e != cudaSuccess) return fail(DF_ECUDA, "autotune: %s", cudaGetErrorString(e));
  return DF_OK;
}

// Autotuner: first the tile shape of every (op, direction) -- each shape timed on
// one coarse step of `runs`, the fastest kept -- then, when tune_grid, the
// persistent blocks per SM of every op with those tiles.  The runs' state is
// restored afterwards, so tuning does not advance them.
int autotune(const std::vector<Run*>& runs, Exec& x, int prec, int transport, TileTable& tiles,
             bool tune_grid, bool single_fast) {
  Snapshot sn;
  int rc = snapshot(runs, sn);
  if (rc) return rc;
  double best[OP_COUNT][3], per[OP_COUNT][3];
  for (int o = 0; o < OP_COUNT; ++o)
    for (int d = 0; d < 3; ++d) best[o][d] = INFINITY;
  TileTable chosen = tiles;
  for (int tk = 0; tk < kNumTiles && !rc; ++tk) {
    TileTable tt;
    for (int o = 0; o < OP_COUNT; ++o)
      for (int d = 0; d < 3; ++d) tt.t[o][d] = tk;
    Plan p;
    p.al = runs.empty() ? Allocator() : runs[0]->al;
    rc = build_plan(p, runs, prec, 0, tt, transport, !single_fast);
    if (!rc) rc = time_plan(p, x, prec, 0, single_fast, per);
    plan_free(p);
    for (int o = 0; o < OP_COUNT && !rc; ++o)
      for (int d = 0; d < 3 && is_box_op(o); ++d)
        if (per[o][d] > 0 && per[o][d] < best[o][d]) {
          best[o][d] = per[o][d];
          chosen.t[o][d] = tk;
        }
  }
  if (!rc) tiles = chosen;
  if (!rc && tune_grid) {
    const int cand[] = {1, 2, 4, 8, 16, 32};
    double best_g[OP_COUNT];
    int best_bps[OP_COUNT];
    for (int o = 0; o < OP_COUNT; ++o) {
      best_g[o] = INFINITY;
      best_bps[o] = x.bps[o];
    }
    Plan p;
    p.al = runs.empty() ? Allocator() : runs[0]->al;
    rc = build_plan(p, runs, prec, 0, tiles, transport, !single_fast);
    for (int gi = 0; gi < 6 && !rc; ++gi) {
      rc = time_plan(p, x, prec, cand[gi], single_fast, per);
      for (int o = 0; o < OP_COUNT && !rc; ++o) {
        double s = per[o][0] + per[o][1] + per[o][2];
        if (s > 0 && s < best_g[o]) {
          best_g[o] = s;
          best_bps[o] = cand[gi];
        }
      }
    }
    plan_free(p);
    if (!rc)
      for (int o = 0; o < OP_COUNT; ++o) x.bps[o] = best_bps[o];
  }
  int rc2 = restore(runs, sn);
  return rc ? rc : rc2;
}

int step_plan(Plan& p, Exec& x, int prec, int n) {
  return prec == DF_FP64 ? plan_step<double>(p, x, n) : plan_step<float>(p, x, n);
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
  return df_create_ground(out, n_levels, n, n, lo, hi, G, precision, device, stream);
}

}  // extern "C"

namespace {

int create_ctx(df_ctx** out, int n_levels, const int n0[3], const int n[3], const double lo[3],
               const double hi[3], int G, int precision, int device, void* stream,
               const Allocator& al) {
  if (!out || !n0 || !n || !lo || !hi) return fail(DF_EINVAL, "null argument");
  *out = nullptr;
  int rc = check_shape(n_levels, n0, n, lo, hi, G, precision);  // before touching the device
  if (rc) return rc;
  CK(cudaSetDevice(device));
  df_ctx* c = new (std::nothrow) df_ctx;
  if (!c) return fail(DF_ENOMEM, "host allocation");
  c->device = device;
  c->user = (cudaStream_t)stream;
  rc = run_create(&c->run, n_levels, n0, n, lo, hi, G, precision, al);
  if (rc) {
    delete c;
    return rc;
  }
  c->plan.al = c->run->al;
  if (!exec_init(c->x, device) ||
      cudaStreamCreateWithFlags(&c->x.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    run_free(c->run);
    delete c;
    return fail(DF_ECUDA, "stream/event creation failed");
  }
  *out = c;
  return DF_OK;
}

}  // namespace

extern "C" {

int df_create_ground(df_ctx** out, int n_levels, const int n0[3], const int n[3],
                     const double lo[3], const double hi[3], int G, int precision, int device,
                     void* stream) {
  return create_ctx(out, n_levels, n0, n, lo, hi, G, precision, device, stream, g_allocator);
}

int df_create_levels(df_ctx** out, int n_levels, int N, const double coarse_lo[3],
                     const double coarse_hi[3], int precision, int device, void* stream,
                     df_alloc_fn alloc, df_free_fn dealloc, void* user) {
  if ((alloc == nullptr) != (dealloc == nullptr))
    return fail(DF_EINVAL, "alloc and dealloc are given together");
  Allocator al = g_allocator;
  if (alloc) {
    al.alloc = alloc;
    al.dealloc = dealloc;
    al.user = user;
  }
  const int n[3] = {N, N, N};
  return create_ctx(out, n_levels, n, n, coarse_lo, coarse_hi, DF_DEFAULT_GHOST, precision,
                    device, stream, al);
}

int df_set_params(df_ctx* c, const df_params* p) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (check_params(p)) return DF_EINVAL;
  if (check_mirror(c->run->nl, c->run->lo, p)) return DF_EINVAL;
  DevGuard g(c->device);
  enter(c);
  int rc = DF_OK;
  c->x.launches += run_set_params(c->run, p, c->x.st, &rc);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->x.st));
  leave(c);
  plan_invalidate(c->plan);
  return rc;
}

int df_step(df_ctx* c, int n, double* t_out) {
  if (check_ctx(c)) return DF_EINVAL;
  if (n < 0) return fail(DF_EINVAL, "negative step count");
  if (n == 0) return t_out ? df_status(c, t_out, nullptr, nullptr) : DF_OK;
  Run* r = c->run;
  if (r->P.dt_fixed <= 0.0 && r->P.hydro_on == 0 && !(r->P.chi > 0.0))
    return fail(DF_EINVAL, "no time-step limit: set dt_fixed, hydro_on or chi");
  DevGuard g(c->device);
  enter(c);
  int rc = DF_OK;
  std::vector<Run*> runs{r};
  // fixed sub-cycling and the Eq. 55-56 search share one plan (xi = 2 everywhere;
  // the search drops second sub-cycles on the device), replayed from a graph
  for (int l = 0; l < r->nl; ++l) r->xi[l] = 2;
  if (!c->plan.valid)
    rc = build_plan(c->plan, runs, r->prec, c->full_boxes, c->tiles, c->transport, false);
  if (!rc) rc = step_plan(c->plan, c->x, r->prec, n);
  leave(c);
  r->stepped = true;
  if (!rc && t_out) {
    const int health = sync_health(c->x.st, r);
    DevScalars h;
    CK(cudaMemcpy(&h, r->ds, sizeof h, cudaMemcpyDeviceToHost));
    *t_out = h.t;
    rc = health;
  }
  return rc;
}

int df_status(df_ctx* c, double* t, double* dt_last, int* unhealthy) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  CK(cudaStreamSynchronize(c->x.st));
  DevScalars h;
  CK(cudaMemcpy(&h, c->run->ds, sizeof h, cudaMemcpyDeviceToHost));
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
  std::vector<std::pair<int, int>> ops;
  for (int l = 0; l < c->run->nl; ++l) ops.push_back({OP_FORCE_LEVEL, l});
  ops.push_back({OP_FORCE_FINAL, 0});
  int rc = run_ops_now(c->run, c->x, ops);
  leave(c);
  if (rc) return rc;
  DevScalars h;
  CK(cudaMemcpy(&h, c->run->ds, sizeof h, cudaMemcpyDeviceToHost));
  for (int d = 0; d < 3; ++d) F[d] = h.F[d];
  return DF_OK;
}

int df_force(df_ctx* c, double F[3], double* along) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!F) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  Run* r = c->run;
  int rc;
  if (!r->stepped) {
    rc = df_force_now(c, F);
    if (rc) return rc;
  } else {
    rc = sync_health(c->x.st, r);
    DevScalars h;
    CK(cudaMemcpy(&h, r->ds, sizeof h, cudaMemcpyDeviceToHost));
    for (int d = 0; d < 3; ++d) F[d] = h.F[d];
    if (rc) return rc;
  }
  if (along) {
    double nv = std::sqrt(r->P.V[0] * r->P.V[0] + r->P.V[1] * r->P.V[1] + r->P.V[2] * r->P.V[2]);
    *along = nv > 0 ? -(F[0] * r->P.V[0] + F[1] * r->P.V[1] + F[2] * r->P.V[2]) / nv : 0.0;
  }
  return DF_OK;
}

int df_compute_dt(df_ctx* c, double* dt, double* dt_level) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  Run* r = c->run;
  enter(c);
  for (int l = 0; l < r->nl; ++l) r->xi[l] = 2;
  DevScalars before;
  CK(cudaMemcpyAsync(&before, r->ds, sizeof before, cudaMemcpyDeviceToHost, c->x.st));
  CK(cudaStreamSynchronize(c->x.st));
  std::vector<std::pair<int, int>> ops;
  for (int l = 0; l < r->nl; ++l) ops.push_back({OP_DT_LEVEL, l});
  ops.push_back({OP_DT_FINAL, 0});
  int rc = run_ops_now(r, c->x, ops);
  if (rc) return rc;
  DevScalars after;
  CK(cudaMemcpy(&after, r->ds, sizeof after, cudaMemcpyDeviceToHost));
  // keep the last coarse step taken (df_status reports it)
  CK(cudaMemcpy(&r->ds->dt, &before.dt, sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(r->ds->dtl, before.dtl, sizeof before.dtl, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(r->ds->dtf, before.dtf, sizeof before.dtf, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(r->ds->dtd, before.dtd, sizeof before.dtd, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(&r->ds->xi1, &before.xi1, sizeof before.xi1, cudaMemcpyHostToDevice));
  leave(c);
  if (dt) *dt = after.dt;
  if (dt_level)
    for (int l = 0; l < r->nl; ++l) dt_level[l] = after.dtlev[l];
  return DF_OK;
}

int df_get_field(df_ctx* c, int level, int field, double* out) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  enter(c);
  int r = io(c->run, c->x.st, level, field, out, nullptr, 0, false, &c->x.launches);
  leave(c);
  return r;
}

int df_set_field(df_ctx* c, int level, int field, const double* in) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  DevGuard g(c->device);
  enter(c);
  int r = io(c->run, c->x.st, level, field, nullptr, in, 0, false, &c->x.launches);
  leave(c);
  return r;
}

int df_get_full(df_ctx* c, int level, int field, double* out) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  DevGuard g(c->device);
  enter(c);
  int r = io(c->run, c->x.st, level, field, out, nullptr, 1, false, &c->x.launches);
  leave(c);
  return r;
}

int df_set_full(df_ctx* c, int level, int field, const double* in) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  DevGuard g(c->device);
  enter(c);
  int r = io(c->run, c->x.st, level, field, nullptr, in, 1, false, &c->x.launches);
  leave(c);
  return r;
}

size_t df_state_size(const df_ctx* c) {
  if (!c || !c->run) return 0;
  return (size_t)c->run->nl * 5 * c->run->nc_max;
}

int df_get_state(df_ctx* c, double* out, double* t_out) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!out) return fail(DF_EINVAL, "null output");
  Run* r = c->run;
  size_t nc = r->nc_max;
  DevGuard g(c->device);
  enter(c);
  for (int l = 0; l < r->nl; ++l)
    for (int f = 0; f < 5; ++f) {
      int rc = io(r, c->x.st, l, f, out + (l * 5 + f) * nc, nullptr, 1, true, &c->x.launches);
      if (rc) return rc;
    }
  leave(c);
  if (t_out) return df_status(c, t_out, nullptr, nullptr);
  return DF_OK;
}

int df_set_state(df_ctx* c, const double* in, double t) {
  if (check_ctx(c)) return DF_EINVAL;
  if (!in) return fail(DF_EINVAL, "null input");
  Run* r = c->run;
  size_t nc = r->nc_max;
  DevGuard g(c->device);
  enter(c);
  for (int l = 0; l < r->nl; ++l)
    for (int f = 0; f < 5; ++f) {
      int rc = io(r, c->x.st, l, f, nullptr, in + (l * 5 + f) * nc, 1, true, &c->x.launches);
      if (rc) return rc;
    }
  leave(c);
  CK(cudaMemcpy(&r->ds->t, &t, sizeof(double), cudaMemcpyHostToDevice));
  int zero = 0;
  CK(cudaMemcpy(&r->ds->unhealthy, &zero, sizeof(int), cudaMemcpyHostToDevice));
  r->stepped = false;
  return DF_OK;
}

int df_prolong(df_ctx* c, int cl) {
  if (check_ctx(c, false)) return DF_EINVAL;
  if (cl < 0 || cl + 1 >= c->run->nl) return fail(DF_EINVAL, "no level below %d", cl);
  DevGuard g(c->device);
  enter(c);
  int rc = run_ops_now(c->run, c->x, {{OP_COMMUP, cl}});
  leave(c);
  return rc;
}

int df_restrict(df_ctx* c, int cl) {
  if (check_ctx(c)) return DF_EINVAL;
  if (cl < 0 || cl + 1 >= c->run->nl) return fail(DF_EINVAL, "no level below %d", cl);
  DevGuard g(c->device);
  enter(c);
  int rc = run_ops_now(c->run, c->x, {{OP_COMMMEAN, cl}});
  leave(c);
  return rc;
}

int df_fill_bc(df_ctx* c) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  enter(c);
  int rc = run_ops_now(c->run, c->x, {{OP_BC, 0}});
  leave(c);
  return rc;
}

long long df_kernel_launches(const df_ctx* c) { return c ? c->x.launches : -1; }

int df_set_timing(df_ctx* c, int on) {
  if (!c) return fail(DF_EINVAL, "null context");
  DevGuard g(c->device);
  harvest_timing(c->x);
  c->x.timing = on != 0;
  for (int k = 0; k < K_NKINDS; ++k) {
    c->x.k_ms[k] = 0.0;
    c->x.k_n[k] = 0;
  }
  return DF_OK;
}

int df_kernel_time(df_ctx* c, int kind, double* ms, long long* launches) {
  if (!c || kind < 0 || kind >= K_NKINDS) return fail(DF_EINVAL, "bad timing query");
  DevGuard g(c->device);
  harvest_timing(c->x);
  if (ms) *ms = c->x.k_ms[kind];
  if (launches) *launches = c->x.k_n[kind];
  return DF_OK;
}

const char* df_kernel_name(int kind) {
  static const char* names[K_NKINDS] = {
      "bc_fill",  "source",   "compress_lum", "diffuse",  "frontier_diff", "tprep",
      "tflux",    "tfrontier", "tmom",        "tupdate",  "vrec_source",   "commup",
      "commmean", "dt",       "force",        "sweep",    "viscosity",     "other"};
  return kind >= 0 && kind < K_NKINDS ? names[kind] : "";
}

int df_autotune(df_ctx* c, int* tiles_out) {
  if (check_ctx(c)) return DF_EINVAL;
  DevGuard g(c->device);
  CK(cudaStreamSynchronize(c->x.st));
  std::vector<Run*> runs{c->run};
  for (int l = 0; l < c->run->nl; ++l) c->run->xi[l] = 2;
  int rc = autotune(runs, c->x, c->run->prec, c->transport, c->tiles, false, true);
  if (rc) return rc;
  if (tiles_out)
    for (int o = 0; o < OP_COUNT; ++o)
      for (int d = 0; d < 3; ++d) tiles_out[3 * o + d] = c->tiles.t[o][d];
  plan_invalidate(c->plan);
  return DF_OK;
}

int set_shapes(TileTable& t, const int* shapes) {
  if (!shapes) return fail(DF_EINVAL, "null argument");
  for (int i = 0; i < 3 * OP_COUNT; ++i)
    if (shapes[i] < 0 || shapes[i] >= kNumTiles) return fail(DF_EINVAL, "bad tile shape %d", shapes[i]);
  for (int o = 0; o < OP_COUNT; ++o)
    for (int d = 0; d < 3; ++d) t.t[o][d] = shapes[3 * o + d];
  return DF_OK;
}

int df_set_tile_shapes(df_ctx* c, const int* shapes) {
  if (check_ctx(c)) return DF_EINVAL;
  int rc = set_shapes(c->tiles, shapes);
  if (!rc) plan_invalidate(c->plan);
  return rc;
}

int df_set_transport(df_ctx* c, int mode) {
  if (check_ctx(c)) return DF_EINVAL;
  if (mode < DF_TRANSPORT_AUTO || mode > DF_TRANSPORT_FUSED)
    return fail(DF_EINVAL, "unknown transport mode %d", mode);
  c->transport = mode;
  plan_invalidate(c->plan);
  return DF_OK;
}

int df_debug_full_boxes(df_ctx* c, int on) {
  if (!c) return fail(DF_EINVAL, "null context");
  c->full_boxes = on != 0;
  plan_invalidate(c->plan);
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

int df_check_df64(const double* a_host, const double* b_host, int n, double* worst) {
  if (!a_host || !b_host || !worst || n < 1) return fail(DF_EINVAL, "bad df64 check input");
  double *da = nullptr, *db = nullptr, *dw = nullptr;
  CK(cudaMalloc(&da, n * sizeof(double)));
  CK(cudaMalloc(&db, n * sizeof(double)));
  CK(cudaMalloc(&dw, 8 * sizeof(double)));
  CK(cudaMemcpy(da, a_host, n * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(db, b_host, n * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemset(dw, 0, 8 * sizeof(double)));
  launch_df64_check(da, db, n, dw, nullptr);
  CK(cudaGetLastError());
  CK(cudaMemcpy(worst, dw, 8 * sizeof(double), cudaMemcpyDeviceToHost));
  cudaFree(da);
  cudaFree(db);
  cudaFree(dw);
  return DF_OK;
}

int df_measure_fp64_peak(int device, int repeats, double* tflops, double* ms_best) {
  if (!tflops || repeats < 1) return fail(DF_EINVAL, "bad FP64 probe arguments");
  CK(cudaSetDevice(device));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  double* sink = nullptr;
  CK(cudaMalloc(&sink, sizeof(double)));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const int blocks = 8 * sms, iters = 4096;  // 8 blocks of 256 threads fill an SM
  long long flops = launch_dfma_probe(blocks, iters, sink, nullptr);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < repeats; ++r) {
    CK(cudaEventRecord(a, nullptr));
    launch_dfma_probe(blocks, iters, sink, nullptr);
    CK(cudaEventRecord(b, nullptr));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  *tflops = (double)flops / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return DF_OK;
}

int df_destroy(df_ctx* c) {
  if (!c) return DF_OK;
  DevGuard g(c->device);
  cudaStreamSynchronize(c->x.st);
  plan_free(c->plan);
  exec_free(c->x);
  run_free(c->run);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->x.st) cudaStreamDestroy(c->x.st);
  delete c;
  return DF_OK;
}

// ------------------------------------------------------------------------ pools

size_t df_run_bytes(int n_levels, const int n[3], int G, int precision) {
  return df_run_bytes_ground(n_levels, n, n, G, precision);
}

size_t df_run_bytes_ground(int n_levels, const int n0[3], const int n[3], int G, int precision) {
  if (!n0 || !n || n_levels < 1 || n_levels > DF_MAX_LEVELS || G < 0) return 0;
  return run_bytes(n_levels, n0, n, G, precision);
}

int df_set_allocator(df_alloc_fn alloc, df_free_fn dealloc, void* user) {
  if ((alloc == nullptr) != (dealloc == nullptr))
    return fail(DF_EINVAL, "alloc and dealloc are set together");
  g_allocator.alloc = alloc;
  g_allocator.dealloc = dealloc;
  g_allocator.user = alloc ? user : nullptr;
  return DF_OK;
}

int df_pool_create(df_pool** out, size_t budget, int precision, int device, void* stream) {
  if (!out) return fail(DF_EINVAL, "null argument");
  *out = nullptr;
  if (precision != DF_FP64 && precision != DF_FP32_STATE)
    return fail(DF_EINVAL, "unknown precision %d", precision);
  CK(cudaSetDevice(device));
  df_pool* p = new (std::nothrow) df_pool;
  if (!p) return fail(DF_ENOMEM, "host allocation");
  p->device = device;
  p->prec = precision;
  p->budget = budget;
  p->user = (cudaStream_t)stream;
  p->plan.al = g_allocator;
  bool ok = exec_init(p->x, device);
  // every pool launch goes through the work-list kernel, so a run's arithmetic is
  // the same alone in a pool and in any mix of runs (bitwise)
  p->x.single_fast = false;
  if (!ok || cudaStreamCreateWithFlags(&p->x.st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    delete p;
    return fail(DF_ECUDA, "stream/event creation failed");
  }
  *out = p;
  return DF_OK;
}

int df_pool_admit(df_pool* p, int n_levels, const int n[3], const double lo[3],
                  const double hi[3], int G, const df_params* prm, int* slot_out) {
  return df_pool_admit_ground(p, n_levels, n, n, lo, hi, G, prm, slot_out);
}

int df_pool_admit_ground(df_pool* p, int n_levels, const int n0[3], const int n[3],
                         const double lo[3], const double hi[3], int G, const df_params* prm,
                         int* slot_out) {
  if (!p || !n0 || !n || !lo || !hi || !slot_out) return fail(DF_EINVAL, "null argument");
  if (check_params(prm)) return DF_EINVAL;
  int rc = check_shape(n_levels, n0, n, lo, hi, G, p->prec);
  if (rc) return rc;
  if (check_mirror(n_levels, lo, prm)) return DF_EINVAL;
  size_t need = run_bytes(n_levels, n0, n, G, p->prec);
  if (p->used + need > p->budget)
    return fail(DF_EBUSY, "HBM budget: %zu used + %zu needed > %zu", p->used, need, p->budget);
  DevGuard g(p->device);
  Run* r = nullptr;
  rc = run_create(&r, n_levels, n0, n, lo, hi, G, p->prec, g_allocator);
  if (rc) return rc;
  enter(p);
  rc = DF_OK;
  p->x.launches += run_set_params(r, prm, p->x.st, &rc);
  cudaError_t e = cudaStreamSynchronize(p->x.st);
  leave(p);
  if (rc || e != cudaSuccess) {
    run_free(r);
    return rc ? rc : fail(DF_ECUDA, "admission: %s", cudaGetErrorString(e));
  }
  int slot = -1;
  for (size_t i = 0; i < p->slots.size(); ++i)
    if (!p->slots[i]) {
      slot = (int)i;
      break;
    }
  if (slot < 0) {
    slot = (int)p->slots.size();
    p->slots.push_back(nullptr);
  }
  p->slots[slot] = r;
  p->used += r->bytes;
  plan_invalidate(p->plan);
  *slot_out = slot;
  return DF_OK;
}

int df_pool_release(df_pool* p, int slot) {
  if (!p || slot < 0 || slot >= (int)p->slots.size() || !p->slots[slot])
    return fail(DF_EINVAL, "no run in slot %d", slot);
  DevGuard g(p->device);
  cudaStreamSynchronize(p->x.st);
  p->used -= p->slots[slot]->bytes;
  run_free(p->slots[slot]);
  p->slots[slot] = nullptr;
  plan_invalidate(p->plan);
  return DF_OK;
}

int df_pool_step(df_pool* p, int n) {
  if (!p) return fail(DF_EINVAL, "null pool");
  if (n < 0) return fail(DF_EINVAL, "negative step count");
  std::vector<Run*> runs;
  for (Run* r : p->slots)
    if (r) runs.push_back(r);
  if (runs.empty() || n == 0) return DF_OK;
  DevGuard g(p->device);
  int rc = DF_OK;
  if (!p->plan.valid) rc = build_plan(p->plan, runs, p->prec, 0, p->tiles, p->transport, true);
  if (rc) return rc;
  enter(p);
  rc = step_plan(p->plan, p->x, p->prec, n);
  leave(p);
  for (Run* r : runs) r->stepped = true;
  return rc;
}

int df_pool_query(df_pool* p, double* out, int max_slots) {
  if (!p || !out) return fail(DF_EINVAL, "null argument");
  DevGuard g(p->device);
  CK(cudaStreamSynchronize(p->x.st));
  int ns = std::min((int)p->slots.size(), max_slots);
  std::vector<DevScalars> h(ns);
  for (int i = 0; i < ns; ++i)
    if (p->slots[i])
      CK(cudaMemcpyAsync(&h[i], p->slots[i]->ds, sizeof(DevScalars), cudaMemcpyDeviceToHost,
                         p->x.st));
  CK(cudaStreamSynchronize(p->x.st));
  for (int i = 0; i < ns; ++i) {
    double* o = out + 6 * i;
    if (!p->slots[i]) {
      for (int k = 0; k < 6; ++k) o[k] = NAN;
      continue;
    }
    o[0] = h[i].F[0];
    o[1] = h[i].F[1];
    o[2] = h[i].F[2];
    o[3] = h[i].t;
    o[4] = h[i].dt;
    o[5] = h[i].unhealthy;
  }
  return ns;
}

int df_pool_force(df_pool* p, int slot, double F_out[3], double* t_out) {
  if (!p || slot < 0 || slot >= (int)p->slots.size() || !p->slots[slot] || !F_out)
    return fail(DF_EINVAL, "no run in slot %d, or a null output", slot);
  DevGuard g(p->device);
  CK(cudaStreamSynchronize(p->x.st));
  DevScalars h;
  CK(cudaMemcpy(&h, p->slots[slot]->ds, sizeof h, cudaMemcpyDeviceToHost));
  for (int d = 0; d < 3; ++d) F_out[d] = h.F[d];
  if (t_out) *t_out = h.t;
  return h.unhealthy ? fail(DF_EUNHEALTHY, "slot %d: NaN, rho <= 0 or e <= 0", slot) : DF_OK;
}

int df_pool_history(df_pool* p, int slot, int k, double* out, int* got) {
  if (!p || slot < 0 || slot >= (int)p->slots.size() || !p->slots[slot] || !out || !got ||
      k < 0)
    return fail(DF_EINVAL, "no run in slot %d, or a bad output", slot);
  Run* r = p->slots[slot];
  DevGuard g(p->device);
  CK(cudaStreamSynchronize(p->x.st));
  long long pos = 0;
  CK(cudaMemcpy(&pos, r->ring_pos, sizeof pos, cudaMemcpyDeviceToHost));
  const long long m = std::min<long long>(std::min<long long>(k, pos), r->ring_cap);
  long long done = 0;
  while (done < m) {  // at most two contiguous pieces of the ring
    const long long e = pos - m + done, at = e % r->ring_cap;
    const long long len = std::min(m - done, r->ring_cap - at);
    CK(cudaMemcpy(out + kRingStride * done, r->ring + kRingStride * at,
                  kRingStride * len * sizeof(double), cudaMemcpyDeviceToHost));
    done += len;
  }
  *got = (int)m;
  return DF_OK;
}

int df_pool_get_field(df_pool* p, int slot, int level, int field, double* out) {
  if (!p || slot < 0 || slot >= (int)p->slots.size() || !p->slots[slot] || !out)
    return fail(DF_EINVAL, "no run in slot %d", slot);
  DevGuard g(p->device);
  enter(p);
  int rc = io(p->slots[slot], p->x.st, level, field, out, nullptr, 0, false, &p->x.launches);
  leave(p);
  return rc;
}

int df_pool_set_field(df_pool* p, int slot, int level, int field, const double* in) {
  if (!p || slot < 0 || slot >= (int)p->slots.size() || !p->slots[slot] || !in)
    return fail(DF_EINVAL, "no run in slot %d", slot);
  DevGuard g(p->device);
  enter(p);
  int rc = io(p->slots[slot], p->x.st, level, field, nullptr, in, 0, false, &p->x.launches);
  leave(p);
  return rc;
}

int df_pool_info(df_pool* p, int* active, size_t* used, size_t* budget, long long* launches) {
  if (!p) return fail(DF_EINVAL, "null pool");
  int a = 0;
  for (Run* r : p->slots)
    if (r) ++a;
  if (active) *active = a;
  if (used) *used = p->used;
  if (budget) *budget = p->budget;
  if (launches) *launches = p->x.launches;
  return DF_OK;
}

int df_pool_set_tiles(df_pool* p, const int* blocks_per_sm) {
  if (!p || !blocks_per_sm) return fail(DF_EINVAL, "null argument");
  for (int o = 0; o < OP_COUNT; ++o)
    if (blocks_per_sm[o] < 1 || blocks_per_sm[o] > 64) return fail(DF_EINVAL, "bad tile setting");
  for (int o = 0; o < OP_COUNT; ++o) p->x.bps[o] = blocks_per_sm[o];
  plan_invalidate(p->plan);
  return DF_OK;
}

int df_pool_set_transport(df_pool* p, int mode) {
  if (!p) return fail(DF_EINVAL, "null pool");
  if (mode < DF_TRANSPORT_AUTO || mode > DF_TRANSPORT_FUSED)
    return fail(DF_EINVAL, "unknown transport mode %d", mode);
  p->transport = mode;
  plan_invalidate(p->plan);
  return DF_OK;
}

int df_pool_set_tile_shapes(df_pool* p, const int* shapes) {
  if (!p) return fail(DF_EINVAL, "null pool");
  int rc = set_shapes(p->tiles, shapes);
  if (!rc) plan_invalidate(p->plan);
  return rc;
}

int df_pool_autotune(df_pool* p, int* blocks_per_sm_out) {
  if (!p) return fail(DF_EINVAL, "null pool");
  std::vector<Run*> runs;
  for (Run* r : p->slots)
    if (r) runs.push_back(r);
  if (runs.empty()) return fail(DF_EINVAL, "empty pool");
  DevGuard g(p->device);
  CK(cudaStreamSynchronize(p->x.st));
  int rc = autotune(runs, p->x, p->prec, p->transport, p->tiles, true, false);
  if (rc) return rc;
  if (blocks_per_sm_out)
    for (int o = 0; o < OP_COUNT; ++o) blocks_per_sm_out[o] = p->x.bps[o];
  plan_invalidate(p->plan);
  return DF_OK;
}

int df_pool_set_timing(df_pool* p, int on) {
  if (!p) return fail(DF_EINVAL, "null pool");
  DevGuard g(p->device);
  harvest_timing(p->x);
  p->x.timing = on != 0;
  for (int k = 0; k < K_NKINDS; ++k) {
    p->x.k_ms[k] = 0.0;
    p->x.k_n[k] = 0;
  }
  return DF_OK;
}

int df_pool_kernel_time(df_pool* p, int kind, double* ms, long long* launches) {
  if (!p || kind < 0 || kind >= K_NKINDS) return fail(DF_EINVAL, "bad timing query");
  DevGuard g(p->device);
  harvest_timing(p->x);
  if (ms) *ms = p->x.k_ms[kind];
  if (launches) *launches = p->x.k_n[kind];
  return DF_OK;
}

int df_pool_destroy(df_pool* p) {
  if (!p) return DF_OK;
  DevGuard g(p->device);
  cudaStreamSynchronize(p->x.st);
  plan_free(p->plan);
  exec_free(p->x);
  for (Run* r : p->slots) run_free(r);
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->ev_out) cudaEventDestroy(p->ev_out);
  if (p->x.st) cudaStreamDestroy(p->x.st);
  delete p;
  return DF_OK;
}

}  // extern "C"
