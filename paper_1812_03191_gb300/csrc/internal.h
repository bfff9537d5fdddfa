// internal.h -- device-side data structures and kernel launchers of libdfnest.
//
// One level (Sec. 3: a mesh is its active cells surrounded by layers of ghost
// cells) is a padded box of s = n + 2G elements per axis, x fastest,
// one structure-of-arrays allocation per field.  rho and e are cell-centred,
// v_d sits on the lower d-face of the cell with the same index.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "df64.h"

namespace dfn {

enum { F_RHO = 0, F_E = 1, F_VX = 2 };

// Everything a kernel needs to know about one level.  Passed by value.
struct LevelView {
  int n[3], G, s[3];
  int st[3];          // element strides (1, s0, s0*s1)
  int nc;             // elements per field
  double dx[3], lo[3], vol, area[3];
  double inv_dx[3], inv_vol, dcoef[3];  // 1/dx, 1/vol, area/dx (diffusion)
  double dt_scale;    // dt of this level = coarse dt * dt_scale
  int off[3];         // lower corner of the active box in the parent's active cells
  void* q[5];         // rho, e, vx, vy, vz
  void* phi;          // potential at cell centres (Eq. 16), in the arithmetic type
  void* lumw;         // luminosity weight / cell volume on active cells, likewise
  double* fw;         // static force weights GM V_c / (r^2 + eps^2)^(3/2), active cells
  double* acc;        // frontier fluxes of this level as a child (CommFlux record, see
                      // rec_index): mass, transported energy, diffused energy; followed
                      // by their sums per coarse slot [side][quantity][slot]
  int acc_slots;      // coarse slots per (side, quantity) of the sums
  // child geometry (coarse frontier overwrite, covered mask), has_child = 0 if none
  int has_child;
  int coff[3], cn[3];
  const double* cacc;  // the child's sums (read by the frontier substitutions)
  int cacc_slots;
  const double* crec;  // the child's record, summed into csum (= cacc) by the parent
  double* csum;
  int is_child;
  // bit d: the lower d-face of the domain is a mirror plane through the perturber
  // (coordinate 0, reflecting) and the run stands for the domain unfolded across it;
  // the same on every level of a run
  int mir;
};

// Scratch shared by all levels of a context (levels are advanced one at a time).
struct Scratch {
  void* pi[3];  // staggered momenta during transport
  void* eps;    // e / rho
  void* w[3];   // Pi / rho_face
  void* F;      // mass flux of the current sweep
  void* E;      // energy flux of the current sweep
  void* P[3];   // momentum fluxes of the current sweep
  // second copy of (rho, e, Pi_x, Pi_y, Pi_z) for the fused sweeps (planes of eps,
  // w and P[0], which the fused path does not use): x writes it, y reads it, z writes it
  void* qb[5];
};

// Box of a stencil op.  tile = 0: elements enumerated x fastest over the box;
// tile = k > 0: in 256-element tiles of tile_extent(k, .) (x, y, z), tiles x
// fastest, so a block's neighbour rows come from its own SM's L1.
struct Box {
  int lo[3], hi[3];
  int tile;
  int zc;  // fused sweeps: planes per chunk of the marching axis
  // flat enumeration: element t -> plane t / (x y extent), row r / (x extent) as
  // multiply-shifts (set by set_divisors; exact for t < 2^31)
  unsigned long long mx, mp;
  int sx, sp;
  long long count() const {
    return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  }
  // q = floor(t / d) = (t m) >> s for every t < 2^31 with s = 31 + ceil(log2 d) and
  // m = ceil(2^s / d): m d = 2^s + e with 0 <= e < d <= 2^(s-31), so
  // t m / 2^s = t / d + t e / (d 2^s) and t e < 2^s keeps the error below 1 / d, too
  // small to carry the quotient over an integer (Granlund & Montgomery, PLDI 1994)
  static void magic(unsigned d, unsigned long long& m, int& s) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    s = 31 + l;
    m = ((1ull << s) + d - 1) / d;
  }
  void set_divisors() {
    const unsigned bx = (unsigned)(hi[0] - lo[0]), by = (unsigned)(hi[1] - lo[1]);
    magic(bx > 0 ? bx : 1u, mx, sx);
    magic(bx * by > 0 ? bx * by : 1u, mp, sp);
  }
};

constexpr int kNumTiles = 5;
// tile extents (x, y, z) with x*y*z = 256 of shape k (k = 0: flat enumeration)
__host__ __device__ inline int tile_extent(int k, int axis) {
  switch (k) {
    case 1: return axis == 0 ? 32 : (axis == 1 ? 8 : 1);
    case 2: return axis == 0 ? 32 : (axis == 1 ? 1 : 8);
    case 3: return axis == 0 ? 32 : (axis == 1 ? 4 : 2);
    case 4: return axis == 0 ? 64 : (axis == 1 ? 4 : 1);
    default: return 1;
  }
}

// Fused transport sweep: a block of kSweepRows + 1 warps; each warp holds one row
// of 32 consecutive x positions (a few of them halo for the x-stencil), the extra
// warp the row below the block's rows, and the block marches through zc planes of
// the marching axis (z for the x sweep, the sweep axis itself for y and z).
constexpr int kSweepRows = 8;
constexpr int kSweepThreads = 32 * (kSweepRows + 1);
__host__ __device__ inline int sweep_own_x(int d) { return d == 0 ? 27 : 31; }
__host__ __device__ inline int sweep_row_axis(int d) { return d == 1 ? 2 : 1; }
__host__ __device__ inline int sweep_march_axis(int d) { return d == 0 ? 2 : d; }
__host__ __device__ inline int sweep_units(const Box& b, int d) {
  const int ra = sweep_row_axis(d), mu = sweep_march_axis(d), ow = sweep_own_x(d);
  const int nsx = (b.hi[0] - b.lo[0] + ow - 1) / ow;
  const int nsr = (b.hi[ra] - b.lo[ra] + kSweepRows - 1) / kSweepRows;
  return nsx * nsr * ((b.hi[mu] - b.lo[mu] + b.zc - 1) / b.zc);
}

struct Phys {
  double gamma, rho0, e0, V[3], GM, eps, chi, L, cfl, cfl_diff, dt_fixed, av_c2;
  double mult;  // copies of the simulated part in the unfolded domain (2^mirror planes)
  int diff_face_rho, hydro_on, band;
  int bc[6];
};

// Device scalars of a context.
// doubles per entry of a run's force history: F_x, F_y, F_z, t at the end of the step
constexpr int kRingStride = 4;

// the constants of a level step, DevScalars::kd / kf [level][K_* + axis]
enum { K_ADT = 0, K_DTDX = 3, K_DIFF = 6, K_F0 = 9 };

struct DevScalars {
  double dt;                  // current coarse step
  double t;                   // simulated time
  double F[3];                // force after the last coarse step
  double dt_last;             // coarse step of the last completed coarse step
  unsigned long long dtmin[48];  // per-level, per-axis max of cs + |v_d| (bit patterns)
  double dtlev[16];              // per-level limits of the last reduction
  double dtl[16];                // level step of each level: dt / prod_{m<l} xi_m
  float dtf[16];                 // the same in FP32
  df64 dtd[16];                  // and in double-float
  // per level, the constants of its level step in the arithmetic types, each the
  // product of its factor (DtFinal::kfac) and the level step, per axis d: A_d dt,
  // dt / dx_d, -chi dt A_d / dx_d (diffusion), rho0 V_d A_d dt (background mass flux)
  df64 kd[16][12];
  float kf[16][12];
  int unhealthy;
  unsigned xi1;  // bit m set when the Eq. 55-56 search chose xi_m = 1 this coarse step
};

// Arithmetic type of the stencils of a state type: the FP32 state computes in float;
// the FP64 state in double-float (df64.h), 48-bit significands on the FP32 pipe,
// since GB300's FP64 pipe runs at 1/64 of its FP32 rate.  Reductions (time step,
// force, frontier flux sums) and the inter-level operators stay in the state type or
// FP64.
template <class T>
struct ArithOf {
  using type = T;
};
template <>
struct ArithOf<double> {
  using type = df64;
};
template <class T>
using Arith = typename ArithOf<T>::type;

// Storage type of the state fields: float for the FP32 state; for the FP64 state a
// double-float pair whose value is a double (df64.h, dstate), 8 bytes like a double,
// which the stencils load and store without conversion.
template <class T>
struct StateOf {
  using type = T;
};
template <>
struct StateOf<double> {
  using type = dstate;
};
template <class T>
using St = typename StateOf<T>::type;

// a double constant in an arithmetic type (host side)
template <class C>
inline C to_arith(double x) {
  return (C)x;
}
template <>
inline df64 to_arith<df64>(double x) {
  return to_df64(x);
}

// per-level geometry constants in the kernels' arithmetic type (no FP64 work in
// FP32 kernels: GB300's FP64 pipe is 1/64 of its FP32 rate)
template <class C>
struct Geo {
  C inv_dx[3], area[3], inv_vol;
};

template <class C>
inline Geo<C> make_geo(const LevelView& L) {
  Geo<C> g;
  for (int d = 0; d < 3; ++d) {
    g.inv_dx[d] = to_arith<C>(L.inv_dx[d]);
    g.area[d] = to_arith<C>(L.area[d]);
  }
  g.inv_vol = to_arith<C>(L.inv_vol);
  return g;
}

// uniform background of Sec. 3.4 in the kernels' arithmetic type
template <class C>
struct Bg {
  C rho0, e0, eps0, V[3];
};

template <class C>
inline Bg<C> make_bg(const Phys& P) {
  Bg<C> b;
  b.rho0 = to_arith<C>(P.rho0);
  b.e0 = to_arith<C>(P.e0);
  b.eps0 = to_arith<C>(P.e0 / P.rho0);
  for (int d = 0; d < 3; ++d) b.V[d] = to_arith<C>(P.V[d]);
  return b;
}

// constants of the Eq. 55 finalisation of one run
struct DtFinal {
  double prod[16];       // prod_{m<l} xi_m (fixed sub-cycling)
  double diff_lim[16];   // explicit-diffusion limit of each level
  double cfl_dx[16][3];  // cfl * dx_d (0 when hydro is off)
  double cost[16];       // Eq. 56 cost of a level step of each level (cells)
  // per level and axis, the factors of the level step's constants (DevScalars::kd):
  // area_d, 1/dx_d, -chi area_d/dx_d, rho0 V_d area_d
  double kfac[16][12];
  int search;            // 1: choose xi_m in {1, 2} each coarse step (Eq. 55-56)
  int pad;
};

// Ops of the work-list kernel.  Every launch runs one op over a list of work
// items; an item is one (run, level) with its box and its own parameters.
// OP_TFRONTIER and OP_ZERO_ACC are no longer emitted (the CommFlux record replaced
// them); they keep their numbers so that op indices (tile-shape controls, timing
// kinds, the binding's op names) stay stable.
enum Op {
  OP_SOURCE = 0, OP_COMPRESS, OP_FRONTIER_DIFF, OP_DIFFUSE, OP_TPREP, OP_TFLUX, OP_TFRONTIER,
  OP_TMOM, OP_TUPDATE, OP_VREC, OP_BC, OP_COMMUP, OP_COMMMEAN, OP_ZERO_ACC, OP_DT_LEVEL,
  OP_DT_FINAL, OP_FORCE_LEVEL, OP_FORCE_FINAL, OP_TIME, OP_SWEEP, OP_VISC_Q, OP_VISC_V,
  OP_COUNT
};

// ops that enumerate the elements of a box (the ones a tile shape applies to)
__host__ __device__ inline bool is_box_op(int op) {
  return op == OP_SOURCE || op == OP_COMPRESS || op == OP_DIFFUSE || op == OP_TPREP ||
         op == OP_TFLUX || op == OP_TMOM || op == OP_TUPDATE || op == OP_VREC ||
         op == OP_VISC_Q || op == OP_VISC_V;
}

// cells per thread of an op: the FP32 state's kicks, compression and diffusion take
// two (with one they are latency-bound: too few bytes in flight per thread)
__host__ __device__ constexpr int cells_per_thread(int op, int esz) {
  return esz == 4 && (op == OP_COMPRESS || op == OP_DIFFUSE || op == OP_SOURCE ||
                      op == OP_VREC)
             ? 2
             : 1;
}

// CommUp tiles (the kernel's comment in kernels.cu says how they are used): per
// field, the coarse hosts with a fine ghost among their children, as six disjoint
// boxes, each cut into tiles of at most kCuHosts hosts in one host plane.
constexpr int kCuHosts = 256;  // hosts per CommUp tile (the block size), <= 64 a side
constexpr int kCuZ = 396;         // max (tx + 2)(ty + 2) over tx, ty <= 64, tx ty <= 256
constexpr int kCuY = 384;         // max ty (tx + 2) over the same tiles

struct CuBox {
  int x0, y0, z0, ex, ey, ez;  // first host and extents
  int tx, ty, ntx, nty;        // tile size and tiles per plane
};

// host range along an axis: 0 lower ghost hosts, 1 upper ghost hosts, 2 kept hosts,
// 3 all hosts; m = n/2 hosts span the active cells, k0 = 1 on a field's own axis
__host__ __device__ inline void cu_range(int which, int m, int hg, int k0, int& lo, int& e) {
  if (which == 0) {
    lo = -hg;
    e = hg + k0;
  } else if (which == 1) {
    lo = m;
    e = hg;
  } else if (which == 2) {
    lo = k0;
    e = m - k0;
  } else {
    lo = -hg;
    e = m + 2 * hg;
  }
}

// box b (0..5) of the shell of a field whose own axis is sa (-1 for a cell field)
__host__ __device__ inline CuBox cu_box(const int* n, int G, int sa, int b) {
  // x: all, all, all, all, lower, upper; y: all, all, lower, upper, kept, kept;
  // z: lower, upper, then kept
  CuBox B;
  const int hg = G >> 1;
  cu_range(b < 4 ? 3 : b - 4, n[0] >> 1, hg, sa == 0, B.x0, B.ex);
  cu_range(b < 2 ? 3 : b < 4 ? b - 2 : 2, n[1] >> 1, hg, sa == 1, B.y0, B.ey);
  cu_range(b < 2 ? b : 2, n[2] >> 1, hg, sa == 2, B.z0, B.ez);
  if (B.ex <= 0 || B.ey <= 0 || B.ez <= 0) {
    B.ez = 0;
    B.tx = B.ty = 1;
    B.ntx = B.nty = 0;
    return B;
  }
  const int sx = (B.ex + 63) / 64;
  B.tx = (B.ex + sx - 1) / sx;
  int ty = B.ey < 64 ? B.ey : 64;
  if (ty > kCuHosts / B.tx) ty = kCuHosts / B.tx;
  B.nty = (B.ey + ty - 1) / ty;
  B.ty = (B.ey + B.nty - 1) / B.nty;
  B.ntx = (B.ex + B.tx - 1) / B.tx;
  return B;
}

// chunks of one CommUp launch into a fine level
__host__ __device__ inline long long cu_chunks(const int* n, int G) {
  long long c = 0;
  for (int f = 0; f < 5; ++f)
    for (int b = 0; b < 6; ++b) {
      const CuBox B = cu_box(n, G, f >= F_VX ? f - F_VX : -1, b);
      c += (long long)B.ez * B.ntx * B.nty;
    }
  return c;
}

enum ItemFlags {
  FL_WRITE_PI = 1, FL_SS3 = 2, FL_LUM = 4, FL_EPS = 8, FL_DFR = 16, FL_HYDRO = 32,
  FL_FUSED = 64,  // VREC: the transport ran as fused sweeps (state in Scratch::qb)
  FL_EPS_ONLY = 128  // TPREP: e/rho only (the x sweep reads Pi/rho_face - V from v)
};

// One work item.  Plain data, copied to shared memory by the kernel; size a
// multiple of 16 bytes.
template <class T>
struct __align__(16) Item {
  LevelView L;          // the level (coarse level of CommUp / CommMean)
  LevelView F;          // fine level of CommUp / CommMean
  Scratch S;            // the run's scratch
  Box b;                // box of stencil ops
  Bg<Arith<T>> bg;
  Geo<Arith<T>> g;
  const void* dt;       // this level's step, Arith<T>
  const void* kc;       // this level step's constants (DevScalars::kd / kf), Arith<T>
  DevScalars* ds;       // the run's scalars
  const DtFinal* fin;   // OP_DT_FINAL constants
  double* partials;     // force partials (this level's first, or the run's for the final sum)
  double* ring;         // force history
  long long* ring_pos;
  Arith<T> gm1, lum, av;
  Arith<T> gga;         // gamma (gamma - 1), the time step's per-cell factor
  double gg, rho0d, e0d, V[3], dt_fixed;
  int ring_cap, npart, level, band, flags, bc_lo, bc_hi;
  unsigned count;       // index-space size of the item
  unsigned br;          // bit m: inside the second sub-cycle of level m + 1 (skipped
                        // when the search chose xi_m = 1)
  int sub;              // sub-cycle of this level step within its parent step (0, 1)
  int pad_;
};

// CommFlux record of a child level (Sec. 3.2.3): for each axis d, the faces of its
// two frontier planes at every transverse position of the padded array (s_t1 x s_t2,
// so a writer needs no bounds test), per side, quantity (mass, transported energy,
// diffused energy) and sub-cycle.  Axis blocks x, y, z one after the other.
__host__ __device__ inline int rec_index(const int s[3], int d, int side, int q, int sub, int c1,
                                         int c2) {
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  int off = 0;
  if (d >= 1) off += 12 * s[1] * s[2];
  if (d >= 2) off += 12 * s[0] * s[2];
  return off + (((side * 3 + q) * 2 + sub) * s[t2] + c2) * s[t1] + c1;
}

__host__ __device__ inline long long rec_elems(const int s[3]) {
  return 12LL * ((long long)s[1] * s[2] + (long long)s[0] * s[2] + (long long)s[0] * s[1]);
}

// ---- kernels.cu: all asynchronous on `st`; return the number of kernels launched.
// host_item (nullable): host copy of the item when nitems == 1; such a launch
// passes the item by value and uses one block per chunk
template <class T>
int launch_batch(int op, int d, const Item<T>* items, const unsigned* starts, int nitems,
                 unsigned nchunks, unsigned grid, cudaStream_t st, const Item<T>* host_item);
int op_chunk_elems(int op, int esz);  // elements per chunk for state elements of esz bytes
int sweep_slots(int esz, int d);      // a context's sweep blocks resident at once
unsigned op_count(int op, int d, const LevelView& L, const LevelView& F, const Box& b);
int force_partials_per_level(const LevelView& L);
int launch_force_weights(const LevelView& L, const Phys& P, cudaStream_t st);
template <class T> int launch_init_uniform(const LevelView& L, const Phys& P, cudaStream_t st);
template <class T> int launch_static_fields(const LevelView& L, const Phys& P, double lum_sigma,
                                            double* wsum, double* partials, cudaStream_t st);
template <class T> int launch_normalise_lum(const LevelView& L, const double* wsum,
                                            double mult, cudaStream_t st);
// host I/O; bgv = background value of the field (0 moves the stored deviations)
template <class T> int launch_pack_active(const LevelView& L, int field, double* out, int full,
                                          double bgv, cudaStream_t st);
template <class T> int launch_unpack_active(const LevelView& L, int field, const double* in,
                                            int full, double bgv, cudaStream_t st);

// kernel kinds for the timing hook (df_kernel_time / df_kernel_name)
enum KernelKind {
  K_BC = 0, K_SOURCE, K_COMPRESS, K_DIFFUSE, K_FRONTIER_DIFF, K_TPREP, K_TFLUX, K_TFRONTIER,
  K_TMOM, K_TUPDATE, K_VREC_SOURCE, K_COMMUP, K_COMMMEAN, K_DT, K_FORCE, K_SWEEP, K_VISC,
  K_OTHER, K_NKINDS
};

// hot-path FP64 division versus IEEE division (device arrays; max_ulp zeroed by caller)
int launch_hdiv_check(const double* a, const double* b, int n, double* max_ulp, cudaStream_t st);
// double-float arithmetic versus FP64 (device arrays; worst[4] zeroed by the caller)
int launch_df64_check(const double* a, const double* b, int n, double* worst, cudaStream_t st);
// launches the FP64 throughput probe; returns the flops it executes
long long launch_dfma_probe(int blocks, int iters, double* sink, cudaStream_t st);

// set the calling thread's last-error message (df_last_error) and return `code`
int set_error(int code, const char* fmt, ...);

}  // namespace dfn
