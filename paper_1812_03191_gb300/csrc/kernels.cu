// kernels.cu -- sm_103a kernels of one level step of the nested-mesh solver
// (Velasco Romero & Masset 2018, Sec. 3) and of the inter-level operators.
//
// Each stencil kernel is one thread per element of a box (flattened, x fastest, so
// consecutive threads touch consecutive addresses).  A kernel applies its operator
// to the elements of the box where its stencil fits inside the padded array; the
// host picks the box (the active cells plus the margin whose values can still reach
// them before the next ghost fill).  T is the state type (double, or float for the
// FP32-state form); time steps, the force and the frontier flux sums are FP64.
//
// The state is stored as deviations from the uniform background of Sec. 3.4:
// drho = rho - rho0, de = e - e0, dv = v - V.  Every flux is written so that its
// background part cancels exactly (the mass flux F' = F - rho0 V_d A dt, etc.);
// the algebra is that of the plain fields, but rounding scales with the
// perturbation instead of the background, which the FP32 state needs (the drag
// is a small difference of large contributions).
#include "internal.h"

#include <math.h>

#include <type_traits>
#include <utility>

namespace dfn {

namespace {

constexpr int kBlock = 256;

// box element t -> (i, j, k); boxes hold fewer than 2^31 elements
__device__ __forceinline__ bool decode(const Box& b, unsigned t, int& i, int& j, int& k) {
  unsigned bx = b.hi[0] - b.lo[0], by = b.hi[1] - b.lo[1], bz = b.hi[2] - b.lo[2];
  if (b.tile == 0) {
    unsigned plane = bx * by;
    if (t >= plane * bz) return false;
    unsigned kk = (unsigned)(((unsigned long long)t * b.mp) >> b.sp);  // t / plane
    unsigned r = t - kk * plane;
    unsigned jj = (unsigned)(((unsigned long long)r * b.mx) >> b.sx);  // r / bx
    i = b.lo[0] + (int)(r - jj * bx);
    j = b.lo[1] + (int)jj;
    k = b.lo[2] + (int)kk;
    return true;
  }
  const unsigned tx = tile_extent(b.tile, 0), ty = tile_extent(b.tile, 1);
  const unsigned tz = tile_extent(b.tile, 2);
  unsigned nx = (bx + tx - 1) / tx, ny = (by + ty - 1) / ty;
  unsigned T = t >> 8, l = t & 255u;
  unsigned Tz = T / (nx * ny), r = T - Tz * nx * ny;
  unsigned Ty = r / nx, Tx = r - Ty * nx;
  unsigned lz = l / (tx * ty), r2 = l - lz * tx * ty;
  unsigned ly = r2 / tx, lx = r2 - ly * tx;
  unsigned ii = Tx * tx + lx, jj = Ty * ty + ly, kk = Tz * tz + lz;
  if (ii >= bx || jj >= by || kk >= bz) return false;
  i = b.lo[0] + (int)ii;
  j = b.lo[1] + (int)jj;
  k = b.lo[2] + (int)kk;
  return true;
}

__device__ __forceinline__ int cidx(const LevelView& L, int i, int j, int k) {
  return (k * L.s[1] + j) * L.s[0] + i;
}

// Division on the hot path.  FP64: one Newton-Raphson refinement of the hardware
// reciprocal estimate (r <- r + r(1 - b r)), then one residual correction
// q <- q + r(a - b q) (Markstein, IBM J. Res. Dev. 34 (1990)): the corrected
// quotient's error is the square of the refined reciprocal's plus the final
// rounding, within one ulp for the normal, non-zero divisors used here (densities,
// 1 + a, and the sum of two same-signed slopes).  FP32: the fast reciprocal-based
// divide.
__device__ __forceinline__ double hdiv(double a, double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  r = fma(r, fma(-b, r, 1.0), r);
  double q = a * r;
  return fma(r, fma(-b, q, a), q);
}
__device__ __forceinline__ float hdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ df64 hdiv(df64 a, df64 b) { return a / b; }
// product and quotient whose result only feeds more arithmetic: in double-float left
// without the final renormalisation (mul_u, div_u in df64.h), in FP32 the plain ones
__device__ __forceinline__ float mul_u(float a, float b) { return a * b; }
__device__ __forceinline__ float div_u(float a, float b) { return __fdividef(a, b); }

// The stencils' arithmetic type C = Arith<T> (internal.h): float for the FP32 state,
// double-float for the FP64 state.  Loads convert the stored value to C, stores round
// C back to the state type.
// The FP64 state is stored as pairs whose values are doubles (dstate, df64.h): loads
// take the pair as it is, stores cut lo onto the pair's grid.
__device__ __forceinline__ float ld(const float* __restrict__ p, int i) { return p[i]; }
__device__ __forceinline__ df64 ld(const df64* __restrict__ p, int i) { return p[i]; }
__device__ __forceinline__ df64 ld(const dstate* __restrict__ p, int i) {
  const dstate v = p[i];
  return df64(v.hi, v.lo);
}
__device__ __forceinline__ void st(df64* p, int i, df64 v) { p[i] = v; }
__device__ __forceinline__ void st(float* p, int i, float v) { p[i] = v; }
__device__ __forceinline__ void st(dstate* p, int i, df64 v) {
  const df64 c = canonical(v);
  p[i] = dstate{c.hi, c.lo};
}
__device__ __forceinline__ bool is0(float v) { return v == 0.f; }
__device__ __forceinline__ bool is0(df64 v) { return v.hi == 0.f; }
// Sums and products with a per-item constant k that is often zero (the background
// wind has one nonzero component): in double-float the operation is skipped when k is
// 0, which gives the same value (a normalised pair plus zero is that pair); in FP32
// the plain expression.  x + k, and x - k y:
__device__ __forceinline__ float add_k(float x, float k) { return k + x; }
__device__ __forceinline__ df64 add_k(df64 x, df64 k) { return k.hi == 0.f ? x : k + x; }
__device__ __forceinline__ float sub_ky(float x, float k, float y) { return x - k * y; }
__device__ __forceinline__ df64 sub_ky(df64 x, df64 k, df64 y) {
  return k.hi == 0.f ? x : x - mul_u(k, y);
}
// k y + z
__device__ __forceinline__ float ky_add(float k, float y, float z) { return k * y + z; }
__device__ __forceinline__ df64 ky_add(df64 k, df64 y, df64 z) {
  return k.hi == 0.f ? z : mul_u(k, y) + z;
}
// e/rho - e0/rho0 of a cell from its deviations, (de - eps0 drho)/(rho0 + drho): one
// expression for every kernel that forms it, so that all give the same bits.  Its
// consumers only take differences of it, so the quotient stays unnormalised.
template <class C, class B>
__device__ __forceinline__ C eps_dev(C de, C dr, const B& bg) {
  return div_u(de - mul_u(bg.eps0, dr), bg.rho0 + dr);
}
// a value as a store of the state keeps it (the FP64 state's stores cut lo)
__device__ __forceinline__ float as_stored(float v) { return v; }
__device__ __forceinline__ df64 as_stored(df64 v) { return canonical(v); }
// two neighbouring elements e, e + 1 (e even) in one vector store
__device__ __forceinline__ void st2(float* p, int e, float a, float b) {
  *reinterpret_cast<float2*>(p + e) = make_float2(a, b);
}
__device__ __forceinline__ void st2(dstate* p, int e, df64 a, df64 b) {
  const df64 ca = canonical(a), cb = canonical(b);
  *reinterpret_cast<float4*>(p + e) = make_float4(ca.hi, ca.lo, cb.hi, cb.lo);
}
// A state value in the state's own type, for the kernels that compute in it (the
// boundary fill, CommMean, the time step, I/O): the float itself, or the exact double
// of a stored pair; put() stores such a value back (a double rounded to the pair).
__device__ __forceinline__ float val(const float* __restrict__ p, int i) { return p[i]; }
__device__ __forceinline__ double val(const dstate* __restrict__ p, int i) {
  return to_double(ld(p, i));
}
__device__ __forceinline__ void put(float* p, int i, float x) { p[i] = x; }
__device__ __forceinline__ void put(dstate* p, int i, double x) { st(p, i, to_df64(x)); }
// exact scalings by 1/2, 2 and other powers of two
__device__ __forceinline__ float pow2_times(float v, float p) { return p * v; }
__device__ __forceinline__ df64 pow2_times(df64 v, float p) { return scale(v, p); }
__device__ __forceinline__ float halve(float v) { return 0.5f * v; }
__device__ __forceinline__ df64 halve(df64 v) { return scale(v, 0.5f); }
__device__ __forceinline__ float twice(float v) { return 2.f * v; }
__device__ __forceinline__ df64 twice(df64 v) { return scale(v, 2.f); }
__device__ __forceinline__ double as_double(float v) { return (double)v; }
__device__ __forceinline__ double as_double(df64 v) { return to_double(v); }
template <class C>
__device__ __forceinline__ C from_double(double x) {
  return (C)x;
}
template <>
__device__ __forceinline__ df64 from_double<df64>(double x) {
  return to_df64(x);
}

// sign tests of the arithmetic types (double-float: df64.h)
__device__ __forceinline__ bool gt0(float v) { return v > 0.f; }
__device__ __forceinline__ bool le0(float v) { return v <= 0.f; }
__device__ __forceinline__ bool lt0(float v) { return v < 0.f; }

// Half the van Leer (1977) harmonic limited slope (Sec. 3.2.1 cites it for the
// interpolation): dl dr / (dl + dr) where dl dr > 0, else 0.  Callers fold the
// factor 2 into their coefficients; scaling by 2 is exact, so the results equal
// those of the full slope bit for bit.  When the product underflows to zero the
// slope is zero, so the divisor dl + dr is never zero or subnormal.  The product and
// the quotient stay unnormalised (mul_u, div_u): the slope only feeds more arithmetic.
template <class C>
__device__ __forceinline__ C hslope(C dl, C dr) {
  C pr = mul_u(dl, dr);
  return le0(pr) ? C(0.f) : div_u(pr, dl + dr);
}

// The upwind side's value, slopes and coefficient are selected first, so one limiter
// (one division) serves both flow directions: u > 0 gives qm + (1 - cour)/2 * slope,
// u <= 0 gives q0 + (-1 - cour)/2 * slope = q0 - (1 + cour)/2 * slope, with
// (+-1 - cour)/2 * slope = (+-1 - cour) * hslope.  In double-float the operands of
// the two one-sided differences are selected before subtracting (two subtractions of
// 11 instructions, not three); in FP32 the three differences are formed and the
// results selected, which measured faster in the fused sweeps (the same values).
template <class C>
__device__ __forceinline__ C upwind_v(C qmm, C qm, C q0, C qp, C u, C cour) {
  const bool up = gt0(u);
  const C a = up ? qm : q0;
  C dl, dr;
  if constexpr (sizeof(C) == 4) {
    const C dm = q0 - qm;
    dl = up ? qm - qmm : dm;
    dr = up ? dm : qp - q0;
  } else {
    dl = a - (up ? qmm : qm);
    dr = (up ? q0 : qp) - a;
  }
  return a + mul_u((up ? C(1.f) : C(-1.f)) - cour, hslope(dl, dr));
}

template <class P, class C>
__device__ __forceinline__ C upwind(const P* __restrict__ q, int c, int s, C u, C cour) {
  return upwind_v(ld(q, c - 2 * s), ld(q, c - s), ld(q, c), ld(q, c + s), u, cour);
}

inline unsigned grid_for(long long n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Programmatic dependent launch: the plan's kernels are launched so that the next
// one is set up while this one drains.  Before touching memory a kernel waits until
// its predecessor has completed and its writes are visible (a no-op for an ordinary
// launch); when a block has done its work it signals that the successor may be
// scheduled.  Stream order is unchanged.  Signalling at the end rather than at the
// start keeps the successor's waiting blocks off the SMs while this grid still runs
// (measured on GB300: signalling at the start slowed the FP64 kernels by 15 % on a
// deep hierarchy of small levels; at the end every workload gained 1-7 %).
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_exit() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// coarse frontier face test: returns side (0/1) and the slot, or -1.  A mirror
// plane is no frontier, and a ghost face across one takes its image's slot.
__device__ __forceinline__ int coarse_frontier(const LevelView& L, int d, int f0, int f1, int f2,
                                               int& slot) {
  int f[3] = {f0, f1, f2};
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  int a = f[t1] - L.G - L.coff[t1], b = f[t2] - L.G - L.coff[t2];
  if (a < 0 && (L.mir >> t1 & 1)) a = -1 - a;
  if (b < 0 && (L.mir >> t2 & 1)) b = -1 - b;
  int h1 = L.cn[t1] >> 1, h2 = L.cn[t2] >> 1;
  if (a < 0 || a >= h1 || b < 0 || b >= h2) return -1;
  int lo = L.G + L.coff[d];
  int side = f[d] == lo && !(L.mir >> d & 1) ? 0 : (f[d] == lo + (L.cn[d] >> 1) ? 1 : -1);
  slot = b * h1 + a;
  return side;
}

// does the low or the high d-face of a cell with d-index gd lie on one of the two
// d-planes that carry the child's frontier faces?
__device__ __forceinline__ bool near_frontier(const LevelView& L, int d, int gd) {
  const int lo = L.G + L.coff[d], hi = lo + (L.cn[d] >> 1);
  return gd == lo || gd == hi || gd + 1 == lo || gd + 1 == hi;
}

// ------------------------------------------------------------------ source S
// S(h) of Eq. 15: v_d -= h [ (p_c - p_m)/(dx rho_face) + (Phi_c - Phi_m)/dx ]
// NC cells per thread (the two-cell form of the compression below): every load of
// all cells first, then the arithmetic and the stores.
template <class T, int NC>
__device__ __forceinline__ void el_source(const LevelView& L, const Box& b, const Scratch& S,
                                          const Arith<T>* __restrict__ dtp, int write_pi,
                                          Arith<T> gm1, const Bg<Arith<T>>& bg,
                                          const Geo<Arith<T>>& g, const unsigned* el) {
  using C = Arith<T>;
  int c[NC], c3[NC][3];
  bool ok[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    int i, j, k;
    ok[n] = decode(b, el[n], i, j, k);
    if (NC == 1 && !ok[n]) return;
    if (!ok[n]) i = j = k = 1;
    c[n] = cidx(L, i, j, k);
    c3[n][0] = i;
    c3[n][1] = j;
    c3[n][2] = k;
  }
  const St<T>* __restrict__ rho = (const St<T>*)L.q[F_RHO];
  const St<T>* __restrict__ e = (const St<T>*)L.q[F_E];
  const Arith<T>* __restrict__ phi = (const Arith<T>*)L.phi;
  const C h = halve(dtp[0]);
  C rc[NC], ec[NC], fc[NC], rm[NC][3], em[NC][3], fm[NC][3], vv[NC][3];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    rc[n] = ld(rho, c[n]);
    ec[n] = ld(e, c[n]);
    fc[n] = ld(phi, c[n]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (c3[n][d] >= 1) {
        const int m = c[n] - L.st[d];
        rm[n][d] = ld(rho, m);
        em[n][d] = ld(e, m);
        fm[n][d] = ld(phi, m);
        vv[n][d] = ld((const St<T>*)L.q[F_VX + d], c[n]);
      }
  }
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    if (!ok[n]) continue;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (c3[n][d] >= 1) {
        C drf = halve(rm[n][d] + rc[n]);
        C rf = bg.rho0 + drf;
        C acc = mul_u(div_u(mul_u(gm1, ec[n] - em[n][d]), rf) + (fc[n] - fm[n][d]),
                      g.inv_dx[d]);
        C vn = vv[n][d] - mul_u(h, acc);
        st((St<T>*)L.q[F_VX + d], c[n], vn);
        // momentum deviation: rf (V + dv) - rho0 V
        if (write_pi)
          st((Arith<T>*)S.pi[d], c[n], mul_u(bg.rho0, vn) + mul_u(drf, add_k(vn, bg.V[d])));
      } else if (write_pi) {
        ((Arith<T>*)S.pi[d])[c[n]] = C(0.f);
      }
    }
  }
}

// ------------------------------------------------------- SubStep2 viscosity
// SubStep2 (Sec. 3.3 stage list, ZEUS naming): the von Neumann-Richtmyer artificial
// viscosity of ZEUS (Stone & Norman 1992).  First pass: along each axis a compressed
// cell (dv = v_d(upper face) - v_d(lower face) < 0) gets q_d = C2 rho dv^2, stored in
// the momentum-flux scratch, and the cell's internal energy loses dt sum_d q_d dv/dx_d
// (from the velocities after the first kick; dv is the same in deviations).
template <class T>
__device__ __forceinline__ void el_visc_q(const LevelView& L, const Box& b, const Scratch& S,
                                          const Arith<T>* __restrict__ dtp, Arith<T> av,
                                          const Bg<Arith<T>>& bg, const Geo<Arith<T>>& g,
                                          unsigned tid) {
  using C = Arith<T>;
  int i, j, k;
  if (!decode(b, tid, i, j, k)) return;
  const int c = cidx(L, i, j, k);
  const int c3[3] = {i, j, k};
  const C rc = bg.rho0 + ld((const St<T>*)L.q[F_RHO], c);
  C heat = C(0.f);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    C q = C(0.f);
    if (c3[d] < L.s[d] - 1) {
      const St<T>* v = (const St<T>*)L.q[F_VX + d];
      const C dv = ld(v, c + L.st[d]) - ld(v, c);
      if (lt0(dv)) q = av * rc * dv * dv;
      heat += q * dv * g.inv_dx[d];
    }
    st((Arith<T>*)S.P[d], c, q);
  }
  St<T>* e = (St<T>*)L.q[F_E];
  st(e, c, ld(e, c) - dtp[0] * heat);
}

// Second pass: v_d -= dt (q_c - q_m) / (dx_d rho_face) on faces 1.. of each axis, and
// the staggered momenta the transport starts from follow the new velocity.
template <class T>
__device__ __forceinline__ void el_visc_v(const LevelView& L, const Box& b, const Scratch& S,
                                          const Arith<T>* __restrict__ dtp, int write_pi,
                                          const Bg<Arith<T>>& bg, const Geo<Arith<T>>& g,
                                          unsigned tid) {
  using C = Arith<T>;
  int i, j, k;
  if (!decode(b, tid, i, j, k)) return;
  const St<T>* __restrict__ rho = (const St<T>*)L.q[F_RHO];
  const int c = cidx(L, i, j, k);
  const int c3[3] = {i, j, k};
  const C dt = dtp[0];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (c3[d] < 1) continue;
    const int m = c - L.st[d];
    const Arith<T>* q = (const Arith<T>*)S.P[d];
    St<T>* v = (St<T>*)L.q[F_VX + d];
    const C drf = halve(ld(rho, m) + ld(rho, c));
    const C vn = ld(v, c) - dt * hdiv(ld(q, c) - ld(q, m), bg.rho0 + drf) * g.inv_dx[d];
    st(v, c, vn);
    if (write_pi) st((Arith<T>*)S.pi[d], c, bg.rho0 * vn + drf * (bg.V[d] + vn));
  }
}

// The compression and diffusion element functions take NC cells per thread: 2 for the
// FP32 state (elements e and e + 256 of a 512-element chunk), 1 otherwise.  Every
// load of both cells is issued before the first store, so a thread keeps twice the
// bytes in flight.  A cell past the end of the box takes an in-bounds stand-in index
// for its loads and stores nothing.  The arithmetic of each cell is unchanged.

// ------------------------------------------------- SubStep3 + luminosity + e/rho
template <class T, int NC>
__device__ __forceinline__ void el_compress_lum(const LevelView& L, const Box& b,
                                                const Scratch& S,
                                                const Arith<T>* __restrict__ dtp, Arith<T> gm1,
                                                Arith<T> lum, int do_ss3, int do_lum, int do_eps,
                                                const Bg<Arith<T>>& bg,
                                                const Geo<Arith<T>>& g, const unsigned* el) {
  using C = Arith<T>;
  int c[NC];
  bool ok[NC], ss3[NC], lm[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    int i, j, k;
    ok[n] = decode(b, el[n], i, j, k);
    if (NC == 1 && !ok[n]) return;
    if (!ok[n]) i = j = k = 0;
    c[n] = cidx(L, i, j, k);
    ss3[n] = do_ss3 && i < L.s[0] - 1 && j < L.s[1] - 1 && k < L.s[2] - 1;
    // active cells and their mirror images in the ghost layers
    lm[n] = do_lum && i >= (L.mir & 1 ? 0 : L.G) && i < L.G + L.n[0] &&
            j >= (L.mir & 2 ? 0 : L.G) && j < L.G + L.n[1] && k >= (L.mir & 4 ? 0 : L.G) &&
            k < L.G + L.n[2];
  }
  St<T>* e = (St<T>*)L.q[F_E];
  const St<T>* vx = (const St<T>*)L.q[F_VX];
  const St<T>* vy = (const St<T>*)L.q[F_VX + 1];
  const St<T>* vz = (const St<T>*)L.q[F_VX + 2];
  C ec[NC], x0[NC], x1[NC], y0[NC], y1[NC], z0[NC], z1[NC], lw[NC], dr[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    ec[n] = ld(e, c[n]);
    if (ss3[n]) {
      x0[n] = ld(vx, c[n]);
      x1[n] = ld(vx, c[n] + L.st[0]);
      y0[n] = ld(vy, c[n]);
      y1[n] = ld(vy, c[n] + L.st[1]);
      z0[n] = ld(vz, c[n]);
      z1[n] = ld(vz, c[n] + L.st[2]);
    }
    if (lm[n]) lw[n] = ld((const Arith<T>*)L.lumw, c[n]);
    if (do_eps) dr[n] = ld((const St<T>*)L.q[F_RHO], c[n]);
  }
  const C dt = dtp[0];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    if (!ok[n]) continue;
    C ecn = ec[n];
    if (ss3[n]) {
      C div = mul_u(x1[n] - x0[n], g.inv_dx[0]) + mul_u(y1[n] - y0[n], g.inv_dx[1]) +
              mul_u(z1[n] - z0[n], g.inv_dx[2]);
      C a = halve(mul_u(mul_u(dt, gm1), div));
      // (e0 + de)(1 - a)/(1 + a) - e0
      ecn = hdiv(mul_u(ecn, C(1.f) - a) - twice(mul_u(a, bg.e0)), C(1.f) + a);
    }
    if (lm[n]) ecn = ecn + mul_u(mul_u(lum, dt), lw[n]);
    st(e, c[n], ecn);
    // e/rho - e0/rho0 = (de - eps0 drho)/(rho0 + drho)
    if (do_eps) st((Arith<T>*)S.eps, c[n], eps_dev(ecn, dr[n], bg));
  }
}

// CommFlux record (Sec. 3.2.3).  A child level writes the flux through each of its
// frontier faces into its record (rec_index), once per sub-cycle; the parent sums the
// entries of a coarse face when it substitutes its own frontier flux, in a fixed
// order: sub-cycle, then the fine faces (u, v) = (0,0), (1,0), (0,1), (1,1).  The
// record is written, never accumulated, so it needs no clearing, and the sub-cycles
// run decide what is summed.

// record a child's flux through the frontier face with index f along d (f = G or
// G + n_d) at transverse position (c1, c2) of the padded array
__device__ __forceinline__ void fr_put(const LevelView& L, int d, int f, int c1, int c2, int q,
                                       int sub, double v) {
  L.acc[rec_index(L.s, d, f == L.G ? 0 : 1, q, sub, c1, c2)] = v;
}

// The parent's substitute for its frontier faces: at the start of its level step
// (in the compression kernel, which every level step that has a consumer runs) one
// thread per (side, quantity, coarse slot) sums the child's record over the
// sub-cycles the child ran (one when the Eq. 55-56 search dropped the second) and
// the 4 fine faces, and the consumers read the sum with one load.
__device__ __forceinline__ void fr_sums(const LevelView& L, const DevScalars* ds, int level,
                                        unsigned tid) {
  if (tid >= 18u * (unsigned)L.cacc_slots) return;
  const int blk = (int)tid / L.cacc_slots, slot = (int)tid - blk * L.cacc_slots;
  const int side = blk / 3, q = blk - 3 * side, d = side >> 1;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int h1 = L.cn[t1] >> 1;
  if (slot >= h1 * (L.cn[t2] >> 1)) return;
  const int a = slot % h1, b = slot / h1;
  const int cs[3] = {L.cn[0] + 2 * L.G, L.cn[1] + 2 * L.G, L.cn[2] + 2 * L.G};
  const bool two = ((ds->xi1 >> level) & 1u) == 0u;
  double sum = 0.0;
  for (int sub = 0; sub < (two ? 2 : 1); ++sub)
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int u = 0; u < 2; ++u)
        sum += L.crec[rec_index(cs, d, side & 1, q, sub, L.G + 2 * a + u, L.G + 2 * b + v)];
  L.csum[blk * L.cacc_slots + slot] = sum;
}


// --------------------------------------------------------------- diffusion
// energy moved in +d across a face during dt: -chi rho_f d(e/rho)/dx * area * dt,
// as rho_f (e/rho difference) K_d with K_d = -chi dt area_d / dx_d, one coefficient
// per level step and axis (a level-step constant) instead of three products per face
template <class T>
__device__ __forceinline__ Arith<T> diff_flux(const LevelView& L, const St<T>* __restrict__ rho,
                                              const Arith<T>* __restrict__ eps, int f, int d,
                                              Arith<T> K, Arith<T> rho0, int dfr) {
  using C = Arith<T>;
  int m = f - L.st[d];
  C rf = dfr ? rho0 : rho0 + halve(ld(rho, m) + ld(rho, f));
  return mul_u(rf, ld(eps, f) - ld(eps, m)) * K;
}

// EPSX: the separate transport kernels follow, and the x sweep's preparation (e/rho
// of the diffused state) is done here: written to Scratch::w[0] (a plane the x sweep
// does not use otherwise; neighbours still read Scratch::eps in this launch), for
// every box cell, from e as stored, so with the bits el_tprep would give.
template <class T, int NC, int EPSX>
__device__ __forceinline__ void el_diffuse(const LevelView& L, const Box& b, const Scratch& S,
                                           const Arith<T>* __restrict__ kc,
                                           Arith<T> rho0, int dfr, const Geo<Arith<T>>& g,
                                           const Bg<Arith<T>>& bg, const unsigned* el) {
  using C = Arith<T>;
  int c[NC], c3[NC][3], ce[NC];
  bool ok[NC], edge[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    int i, j, k;
    const bool in = decode(b, el[n], i, j, k);
    ok[n] = in && i >= 1 && j >= 1 && k >= 1 && i < L.s[0] - 1 && j < L.s[1] - 1 &&
            k < L.s[2] - 1;
    edge[n] = EPSX && in && !ok[n];
    if (NC == 1 && !ok[n] && !edge[n]) return;
    ce[n] = in ? cidx(L, i, j, k) : 0;
    if (!ok[n]) i = j = k = 1;
    c[n] = cidx(L, i, j, k);
    c3[n][0] = i;
    c3[n][1] = j;
    c3[n][2] = k;
  }
  const St<T>* __restrict__ rho = (const St<T>*)L.q[F_RHO];
  const Arith<T>* __restrict__ eps = (const Arith<T>*)S.eps;
  C q[NC][3][2];  // flux through the lower and the upper d-face
#pragma unroll
  for (int n = 0; n < NC; ++n)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const C K = kc[K_DIFF + d];
      q[n][d][0] = diff_flux<T>(L, rho, eps, c[n], d, K, rho0, dfr);
      q[n][d][1] = diff_flux<T>(L, rho, eps, c[n] + L.st[d], d, K, rho0, dfr);
    }
  if (L.has_child) {
#pragma unroll
    for (int n = 0; n < NC; ++n)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!near_frontier(L, d, c3[n][d])) continue;
        int slot, f3[3] = {c3[n][0], c3[n][1], c3[n][2]};
        int side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
        if (side >= 0)
          q[n][d][0] = from_double<C>(L.cacc[((2 * d + side) * 3 + 2) * L.cacc_slots + slot]);
        f3[d] += 1;
        side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
        if (side >= 0)
          q[n][d][1] = from_double<C>(L.cacc[((2 * d + side) * 3 + 2) * L.cacc_slots + slot]);
      }
  }
  St<T>* e = (St<T>*)L.q[F_E];
  C ev[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) ev[n] = ld(e, c[n]);
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    C div = C(0.f);
#pragma unroll
    for (int d = 0; d < 3; ++d) div += q[n][d][1] - q[n][d][0];
    if (ok[n]) {
      const C en = ev[n] - div * g.inv_vol;
      st(e, c[n], en);
      if (EPSX) {
        const C rc = ld(rho, c[n]);
        st((Arith<T>*)S.w[0], c[n], eps_dev(as_stored(en), rc, bg));
      }
    } else if (edge[n]) {
      const C rc = ld(rho, ce[n]);
      st((Arith<T>*)S.w[0], ce[n], eps_dev(ld(e, ce[n]), rc, bg));
    }
  }
}

// CommFlux record of the diffusive energy fluxes through a child's frontier faces:
// one thread per fine frontier face (a launch of its own:
// inside the diffusion kernel the record code would cost that kernel occupancy)
template <class T>
__device__ __forceinline__ void el_frontier_diff(const LevelView& L, const Scratch& S,
                                                 const Arith<T>* __restrict__ kc,
                                                 Arith<T> rho0, int dfr, int sub, unsigned tid) {
  using C = Arith<T>;
  // one thread per fine face: (side, coarse slot, fine face u, v of the slot)
  if (tid >= 24u * (unsigned)L.acc_slots) return;
  const int u = (int)(tid & 1u), v = (int)((tid >> 1) & 1u);
  const int rest = (int)(tid >> 2);
  const int side = rest / L.acc_slots, slot = rest - side * L.acc_slots;
  const int d = side >> 1, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int h1 = L.n[t1] >> 1;
  if (slot >= h1 * (L.n[t2] >> 1)) return;
  const int a = slot % h1, b = slot / h1;
  const int fd = (side & 1) ? L.G + L.n[d] : L.G;
  int f3[3];
  f3[d] = fd;
  f3[t1] = L.G + 2 * a + u;
  f3[t2] = L.G + 2 * b + v;
  const int f = (f3[2] * L.s[1] + f3[1]) * L.s[0] + f3[0];
  fr_put(L, d, fd, f3[t1], f3[t2], 2, sub,
         as_double(diff_flux<T>(L, (const St<T>*)L.q[F_RHO], (const Arith<T>*)S.eps, f, d,
                                kc[K_DIFF + d], rho0, dfr)));
}

// --------------------------------------------------------------- transport
template <class T>
__device__ __forceinline__ void el_tprep(const LevelView& L, const Box& b, const Scratch& S,
                                         const Bg<Arith<T>>& bg, int eps_only, unsigned tid) {
  using C = Arith<T>;
  int i, j, k;
  if (!decode(b, tid, i, j, k)) return;
  const St<T>* __restrict__ rho = (const St<T>*)L.q[F_RHO];
  const int c = cidx(L, i, j, k);
  const int c3[3] = {i, j, k};
  const C rc = ld(rho, c);
  const C ec = ld((const St<T>*)L.q[F_E], c);
  if (eps_only) {
    st((Arith<T>*)S.eps, c, eps_dev(ec, rc, bg));
    return;
  }
  // every load first, then the arithmetic and the stores
  C rm[3], pm[3];
#pragma unroll
  for (int m = 0; m < 3; ++m)
    if (c3[m] >= 1) {
      rm[m] = ld(rho, c - L.st[m]);
      pm[m] = ld((const Arith<T>*)S.pi[m], c);
    }
  C wv[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    wv[m] = C(0.f);
    if (c3[m] >= 1) {
      // Pi/rho_face - V = (dPi - V drf)/(rho0 + drf)
      C drf = halve(rm[m] + rc);
      wv[m] = div_u(sub_ky(pm[m], bg.V[m], drf), bg.rho0 + drf);
    }
  }
  st((Arith<T>*)S.eps, c, eps_dev(ec, rc, bg));
#pragma unroll
  for (int m = 0; m < 3; ++m) st((Arith<T>*)S.w[m], c, wv[m]);
}

// mass and energy flux at d-faces 2 <= i_d < s_d - 1
// the sweep direction is a template parameter: every per-axis constant is then a
// fixed kernel-parameter operand instead of a dynamically indexed load
template <class T, int d>
__device__ __forceinline__ void el_tflux(const LevelView& L, const Box& b, const Scratch& S,
                                         const Arith<T>* __restrict__ kc,
                                         const Bg<Arith<T>>& bg, int sub, unsigned tid) {
  using C = Arith<T>;
  int i, j, k;
  if (!decode(b, tid, i, j, k)) return;
  const int c = cidx(L, i, j, k);
  const int c3[3] = {i, j, k};
  C Fv = C(0.f), Ev = C(0.f);
  if (c3[d] >= 2 && c3[d] < L.s[d] - 1) {
    const int sd = L.st[d];
    const C Adt = kc[K_ADT + d];
    const C du = ld((const St<T>*)L.q[F_VX + d], c);
    const C u = add_k(du, bg.V[d]);
    const C cour = mul_u(u, kc[K_DTDX + d]);
    const C F0 = is0(bg.V[d]) ? C(0.f) : kc[K_F0 + d];
    C drs = upwind((const St<T>*)L.q[F_RHO], c, sd, u, cour);
    Fv = (mul_u(bg.rho0, du) + mul_u(drs, u)) * Adt;  // F - rho0 V_d A dt
    C des = upwind((const Arith<T>*)S.eps, c, sd, u, cour);
    Ev = mul_u(bg.eps0, Fv) + mul_u(des, add_k(Fv, F0));  // E - eps0 rho0 V_d A dt
  }
  st((Arith<T>*)S.F, c, Fv);
  st((Arith<T>*)S.E, c, Ev);
  if (L.is_child && (c3[d] == L.G || c3[d] == L.G + L.n[d])) {  // CommFlux record
    constexpr int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    fr_put(L, d, c3[d], c3[t1], c3[t2], 0, sub, as_double(Fv));
    fr_put(L, d, c3[d], c3[t1], c3[t2], 1, sub, as_double(Ev));
  }
}

// staggered momentum fluxes of sweep d
// staggered momentum fluxes of sweep d (deviation: P - V_m rho0 V_d A dt)
template <class T, int d>
__device__ __forceinline__ void el_tmom(const LevelView& L, const Box& b, const Scratch& S,
                                        const Arith<T>* __restrict__ kc, const Bg<Arith<T>>& bg,
                                        unsigned tid) {
  using C = Arith<T>;
  int i, j, k;
  if (!decode(b, tid, i, j, k)) return;
  const int c = cidx(L, i, j, k);
  const int c3[3] = {i, j, k};
  const int sd = L.st[d];
  const St<T>* __restrict__ vd = (const St<T>*)L.q[F_VX + d];
  const Arith<T>* __restrict__ F = (const Arith<T>*)S.F;
  const C dtdx = kc[K_DTDX + d];
  const C F0 = is0(bg.V[d]) ? C(0.f) : kc[K_F0 + d];
  C Pv[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    C P = C(0.f);
    if (m == d) {
      if (c3[d] >= 2 && c3[d] < L.s[d] - 2) {
        C uc = add_k(halve(ld(vd, c) + ld(vd, c + sd)), bg.V[d]);
        C Fc = halve(ld(F, c) + ld(F, c + sd));
        C ws = d == 0 ? upwind((const St<T>*)S.w[m], c + sd, sd, uc, mul_u(uc, dtdx))
                      : upwind((const Arith<T>*)S.w[m], c + sd, sd, uc, mul_u(uc, dtdx));
        P = ky_add(bg.V[m], Fc, mul_u(ws, add_k(Fc, F0)));
      }
    } else if (c3[d] >= 2 && c3[d] < L.s[d] - 1 && c3[m] >= 1) {
      const int sm = L.st[m];
      C ue = add_k(halve(ld(vd, c - sm) + ld(vd, c)), bg.V[d]);
      C Fe = halve(ld(F, c - sm) + ld(F, c));
      C ws = d == 0 ? upwind((const St<T>*)S.w[m], c, sd, ue, mul_u(ue, dtdx))
                    : upwind((const Arith<T>*)S.w[m], c, sd, ue, mul_u(ue, dtdx));
      P = ky_add(bg.V[m], Fe, mul_u(ws, add_k(Fe, F0)));
    }
    Pv[m] = P;
  }
  // the stores after every load of the three components
#pragma unroll
  for (int m = 0; m < 3; ++m) st((Arith<T>*)S.P[m], c, Pv[m]);
}

// Every load first, then the arithmetic and the stores (a load never waits for a store
// it cannot be reordered with); NC cells per thread as in the compression (one here).
template <class T, int d, int NC>
__device__ __forceinline__ void el_tupdate(const LevelView& L, const Box& b, const Scratch& S,
                                           const Geo<Arith<T>>& g, const unsigned* el) {
  using C = Arith<T>;
  int c[NC], c3[NC][3];
  bool ok[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    int i, j, k;
    ok[n] = decode(b, el[n], i, j, k);
    if (NC == 1 && !ok[n]) return;
    if (!ok[n]) i = j = k = 3;  // an in-bounds stand-in (arrays hold 2 G >= 6 ghosts)
    c[n] = cidx(L, i, j, k);
    c3[n][0] = i;
    c3[n][1] = j;
    c3[n][2] = k;
  }
  const int sd = L.st[d];
  const C iv = g.inv_vol;
  St<T>* rho = (St<T>*)L.q[F_RHO];
  St<T>* e = (St<T>*)L.q[F_E];
  C Flo[NC], Fhi[NC], Elo[NC], Ehi[NC], rv[NC], ev[NC], pv[NC][3], Pa[NC][3], Pb[NC][3];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    Flo[n] = ld((const Arith<T>*)S.F, c[n]);
    Fhi[n] = ld((const Arith<T>*)S.F, c[n] + sd);
    Elo[n] = ld((const Arith<T>*)S.E, c[n]);
    Ehi[n] = ld((const Arith<T>*)S.E, c[n] + sd);
    rv[n] = ld(rho, c[n]);
    ev[n] = ld(e, c[n]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const Arith<T>* P = (const Arith<T>*)S.P[m];
      pv[n][m] = ld((const Arith<T>*)S.pi[m], c[n]);
      Pa[n][m] = ld(P, m == d ? c[n] - sd : c[n]);
      Pb[n][m] = ld(P, m == d ? c[n] : c[n] + sd);
    }
  }
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    if (!ok[n]) continue;
    if (c3[n][d] >= 2 && c3[n][d] < L.s[d] - 2) {
      if (L.has_child && near_frontier(L, d, c3[n][d])) {
        int slot, f3[3] = {c3[n][0], c3[n][1], c3[n][2]};
        int side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
        if (side >= 0) {
          Flo[n] = from_double<C>(L.cacc[((2 * d + side) * 3 + 0) * L.cacc_slots + slot]);
          Elo[n] = from_double<C>(L.cacc[((2 * d + side) * 3 + 1) * L.cacc_slots + slot]);
        }
        f3[d] += 1;
        side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
        if (side >= 0) {
          Fhi[n] = from_double<C>(L.cacc[((2 * d + side) * 3 + 0) * L.cacc_slots + slot]);
          Ehi[n] = from_double<C>(L.cacc[((2 * d + side) * 3 + 1) * L.cacc_slots + slot]);
        }
      }
      st(rho, c[n], rv[n] - (Fhi[n] - Flo[n]) * iv);
      st(e, c[n], ev[n] - (Ehi[n] - Elo[n]) * iv);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const bool chg = m == d ? (c3[n][d] >= 3 && c3[n][d] < L.s[d] - 2)
                              : (c3[n][d] >= 2 && c3[n][d] < L.s[d] - 2 && c3[n][m] >= 1);
      if (chg) st((Arith<T>*)S.pi[m], c[n], pv[n][m] - (Pb[n][m] - Pa[n][m]) * iv);
    }
  }
}

// ------------------------------------------------------- fused transport sweep
// One sweep along d (Sec. 3.1 transport: the mass flux F = rho* v A dt with the
// time-centred van Leer value rho*, e and the momenta carried as (q/rho)* F) with
// the arithmetic of tprep + tflux + tmom + tupdate, fused and register-blocked.
// A block is kSweepRows + 1 warps; warp w holds row row0 - 1 + w (the first is the
// halo row below the block's rows), lane l the x position x0 - hx + l, and the block
// marches through a chunk of planes of the marching axis.  Values along the marching
// axis stay in per-thread registers, x neighbours come by warp shuffle, the row
// below through one shared-memory exchange per plane.
//   y, z sweeps: march along the sweep; the stencil along d is the register window.
//   x sweep: march along z; the stencil along x is a shuffle (3 halo lanes below,
//            2 above), the z neighbour is the previous plane's registers.
// Ping-pong state: the sweep reads `src` inside the box and the level's own arrays
// outside it (the values the separate kernels, which update in place, read there)
// and writes every box cell it owns to `dst`: x and z sweeps from the level's
// arrays to Scratch::qb, the y sweep back.  For a child level the fluxes through
// its frontier faces also go to Scratch::F/E (frontier capture).

__device__ __forceinline__ float shfl_up(float v, int k) {
  return __shfl_up_sync(0xffffffffu, v, k);
}
__device__ __forceinline__ float shfl_dn(float v, int k) {
  return __shfl_down_sync(0xffffffffu, v, k);
}
__device__ __forceinline__ df64 shfl_up(df64 v, int k) {
  return df64(__shfl_up_sync(0xffffffffu, v.hi, k), __shfl_up_sync(0xffffffffu, v.lo, k));
}
__device__ __forceinline__ df64 shfl_dn(df64 v, int k) {
  return df64(__shfl_down_sync(0xffffffffu, v.hi, k), __shfl_down_sync(0xffffffffu, v.lo, k));
}

// coarse-level frontier substitution of the low/high d-face fluxes of cell (g); the
// frontier faces lie on two d-planes, tested first
template <class C>
__device__ __forceinline__ void frontier_fluxes(const LevelView& L, int d, const int g[3], C& Flo,
                                                C& Fhi, C& Elo, C& Ehi) {
  if (!near_frontier(L, d, g[d])) return;
  int slot, f3[3] = {g[0], g[1], g[2]};
  int side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
  if (side >= 0) {
    Flo = from_double<C>(L.cacc[((2 * d + side) * 3 + 0) * L.cacc_slots + slot]);
    Elo = from_double<C>(L.cacc[((2 * d + side) * 3 + 1) * L.cacc_slots + slot]);
  }
  f3[d] += 1;
  side = coarse_frontier(L, d, f3[0], f3[1], f3[2], slot);
  if (side >= 0) {
    Fhi = from_double<C>(L.cacc[((2 * d + side) * 3 + 0) * L.cacc_slots + slot]);
    Ehi = from_double<C>(L.cacc[((2 * d + side) * 3 + 1) * L.cacc_slots + slot]);
  }
}

template <class T, int d>
__device__ __forceinline__ void el_sweep(const Item<T>& it, unsigned unit,
                                         Arith<T>* __restrict__ xch) {
  using C = Arith<T>;
  constexpr int RA = d == 1 ? 2 : 1;  // row axis
  constexpr int MU = d == 0 ? 2 : d;  // marching axis
  constexpr int HX = d == 0 ? 3 : 1;  // halo lanes below the owned x range
  constexpr int OWNX = d == 0 ? 27 : 31;
  constexpr int NT = kSweepThreads;
  constexpr bool kFromB = d == 1;  // x: A -> B, y: B -> A, z: A -> B
  const LevelView& L = it.L;
  const Box& b = it.b;
  const Scratch& S = it.S;
  const Bg<C>& bg = it.bg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nsx = (b.hi[0] - b.lo[0] + OWNX - 1) / OWNX;
  const int nsr = (b.hi[RA] - b.lo[RA] + kSweepRows - 1) / kSweepRows;
  const int cm = (int)unit / (nsx * nsr), crem = (int)unit - cm * nsx * nsr;
  const int sr = crem / nsx, sx = crem - sr * nsx;
  const int x = b.lo[0] + sx * OWNX - HX + lane;
  const int row = b.lo[RA] + sr * kSweepRows - 1 + warp;
  const int m0 = b.lo[MU] + cm * b.zc, m1 = min(m0 + b.zc, b.hi[MU]);
  const int s0 = L.s[0], sRA = L.s[RA], sMU = L.s[MU];
  const int stR = L.st[RA], stM = L.st[MU];
  const bool pos = (unsigned)x < (unsigned)s0 && (unsigned)row < (unsigned)sRA;
  const bool owned = warp >= 1 && lane >= HX && lane < HX + OWNX && x < b.hi[0] &&
                     row < b.hi[RA];
  const bool xrbox = x >= b.lo[0] && x < b.hi[0] && row >= b.lo[RA] && row < b.hi[RA];
  const int cxr = x + row * stR;
  const St<T>* rhoA = (const St<T>*)L.q[F_RHO];
  const St<T>* eA = (const St<T>*)L.q[F_E];
  const St<T>* rhoS = kFromB ? (const St<T>*)S.qb[0] : rhoA;
  const St<T>* eS = kFromB ? (const St<T>*)S.qb[1] : eA;
  const St<T>* __restrict__ vd = (const St<T>*)L.q[F_VX + d];
  St<T>* rhoD = kFromB ? (St<T>*)L.q[F_RHO] : (St<T>*)S.qb[0];
  St<T>* eD = kFromB ? (St<T>*)L.q[F_E] : (St<T>*)S.qb[1];
  // the momenta are scratch (arithmetic type), rho and e the state type in both copies
  const C* piA[3] = {(const C*)S.pi[0], (const C*)S.pi[1], (const C*)S.pi[2]};
  const C* piS[3] = {kFromB ? (const C*)S.qb[2] : piA[0], kFromB ? (const C*)S.qb[3] : piA[1],
                     kFromB ? (const C*)S.qb[4] : piA[2]};
  C* piD[3] = {kFromB ? (C*)S.pi[0] : (C*)S.qb[2], kFromB ? (C*)S.pi[1] : (C*)S.qb[3],
               kFromB ? (C*)S.pi[2] : (C*)S.qb[4]};
  const C dt = ((const C*)it.dt)[0];
  const C Adt = it.g.area[d] * dt;
  const C dtdx = dt * it.g.inv_dx[d];
  const C F0 = bg.rho0 * bg.V[d] * Adt;
  const C iv = it.g.inv_vol;
  const int sd = L.s[d];

  // state of plane p at this thread's (x, row); zero outside the array
  auto load = [&](int p, C& r_, C& e_, C& v_, C (&pi_)[3]) {
    r_ = e_ = v_ = C(0.f);
    pi_[0] = pi_[1] = pi_[2] = C(0.f);
    if (pos && (unsigned)p < (unsigned)sMU) {
      const int c = cxr + p * stM;
      const bool own = !kFromB || (xrbox && p >= b.lo[MU] && p < b.hi[MU]);
      r_ = ld(own ? rhoS : rhoA, c);
      e_ = ld(own ? eS : eA, c);
      v_ = ld(vd, c);
#pragma unroll
      for (int m = 0; m < 3; ++m) pi_[m] = ld(own ? piS[m] : piA[m], c);
    }
  };
  auto gcoord = [&](int p, int (&g)[3]) {
    g[0] = x;
    g[RA] = row;
    g[MU] = p;
  };
  C nr, ne, nv, np[3];

  if constexpr (d != 0) {
    // ================================================= march along the sweep axis
    // windows, oldest first, at step r: rho, eps planes r-3..r; e, v_d, Pi planes
    // r-2..r; w planes r-3..r; F, E faces r-2, r-1; P_d planes r-3, r-2; P_x and
    // P_row planes r-2, r-1.  The update is of plane r - 2.
    constexpr int mx = 0, mr = RA;
    C rw[4] = {}, sw[4] = {}, er[3] = {}, vw[3] = {}, pw[3][3] = {}, ww[3][4] = {};
    C Fw[2] = {}, Ew[2] = {}, Pd[2] = {}, Pm[2][2] = {};
    const int nit = m1 - m0 + 5;
    // Planes far from the array's ends, from the chunk's ends and from a child's
    // frontier planes pass every test on the plane index; their iterations run a
    // copy of the body without those tests (FAST), the others the full one.
    const int r_lo = max(5, m0 + 2), r_hi = min(m1, b.hi[MU] - 2);
    // state of plane p (inside the box and the array) at this thread's (x, row)
    auto load_in = [&](int p, C& r_, C& e_, C& v_, C (&pi_)[3]) {
      r_ = e_ = v_ = C(0.f);
      pi_[0] = pi_[1] = pi_[2] = C(0.f);
      if (pos) {
        const int c = cxr + p * stM;
        const bool own = !kFromB || xrbox;
        r_ = ld(own ? rhoS : rhoA, c);
        e_ = ld(own ? eS : eA, c);
        v_ = ld(vd, c);
#pragma unroll
        for (int m = 0; m < 3; ++m) pi_[m] = ld(own ? piS[m] : piA[m], c);
      }
    };
    auto step = [&](int i, auto fast_tag) {
      constexpr bool FAST = decltype(fast_tag)::value;
      const int r = m0 - 3 + i;
      rw[0] = rw[1]; rw[1] = rw[2]; rw[2] = rw[3]; rw[3] = nr;
      sw[0] = sw[1]; sw[1] = sw[2]; sw[2] = sw[3];
      sw[3] = eps_dev(ne, nr, bg);
      er[0] = er[1]; er[1] = er[2]; er[2] = ne;
      vw[0] = vw[1]; vw[1] = vw[2]; vw[2] = nv;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        pw[m][0] = pw[m][1]; pw[m][1] = pw[m][2]; pw[m][2] = np[m];
      }
      if (FAST)
        load_in(r + 1, nr, ne, nv, np);
      else if (i + 1 < nit)
        load(r + 1, nr, ne, nv, np);
      // mass and energy flux of face plane f = r - 1
      const int f = r - 1;
      C Fv = C(0.f), Evv = C(0.f);
      if (pos && (FAST || (f >= 2 && f < sd - 1))) {
        const C du = vw[1];
        const C u = bg.V[d] + du;
        const C cour = u * dtdx;
        const C drs = upwind_v(rw[0], rw[1], rw[2], rw[3], u, cour);
        Fv = (bg.rho0 * du + drs * u) * Adt;
        const C des = upwind_v(sw[0], sw[1], sw[2], sw[3], u, cour);
        Evv = bg.eps0 * Fv + des * (F0 + Fv);
      }
      Fw[0] = Fw[1]; Fw[1] = Fv;
      Ew[0] = Ew[1]; Ew[1] = Evv;
      if (!FAST && L.is_child && owned && f >= m0 && f < m1 &&
          (f == L.G || f == L.G + L.n[d])) {
        // CommFlux record: transverse axes x and the row axis
        fr_put(L, d, f, x, row, 0, it.sub, as_double(Fv));
        fr_put(L, d, f, x, row, 1, it.sub, as_double(Evv));
      }
      // rho_r, v_{r-1}, F_{r-1} of the row below (shared) and of x - 1 (shuffle)
      C* xb = xch + (i & 1) * 3 * NT;
      xb[tid] = rw[3];
      xb[NT + tid] = vw[1];
      xb[2 * NT + tid] = Fv;
      __syncthreads();
      if (warp == 0) return;  // the halo row only supplies rho, v_d and F
      const C r_rb = xb[tid - 32], v_rb = xb[NT + tid - 32], F_rb = xb[2 * NT + tid - 32];
      const C r_xb = shfl_up(rw[3], 1), v_xb = shfl_up(vw[1], 1), F_xb = shfl_up(Fv, 1);
      // w = (dPi - V drf) / (rho0 + drf) of plane r
      const bool pok = pos && (FAST || (unsigned)r < (unsigned)sMU);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const C rn = m == mx ? r_xb : (m == mr ? r_rb : rw[2]);
        const bool g1 = m == mx ? x >= 1 : (m == mr ? row >= 1 : (FAST || r >= 1));
        C wv = C(0.f);
        if (pok && g1) {
          const C drf = halve(rn + rw[3]);
          wv = hdiv(pw[m][2] - bg.V[m] * drf, bg.rho0 + drf);
        }
        ww[m][0] = ww[m][1]; ww[m][1] = ww[m][2]; ww[m][2] = ww[m][3]; ww[m][3] = wv;
      }
      // P_x, P_row of plane q = r - 1 (d-m edges)
      const int q = r - 1;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int m = j == 0 ? mx : mr;
        C P = C(0.f);
        if (pos && (FAST || (q >= 2 && q < sd - 1)) && (j == 0 ? x >= 1 : row >= 1)) {
          const C ue = bg.V[d] + halve((j == 0 ? v_xb : v_rb) + vw[1]);
          const C Fe = halve((j == 0 ? F_xb : F_rb) + Fv);
          const C wsv = upwind_v(ww[m][0], ww[m][1], ww[m][2], ww[m][3], ue, ue * dtdx);
          P = bg.V[m] * Fe + wsv * (F0 + Fe);
        }
        Pm[j][0] = Pm[j][1];
        Pm[j][1] = P;
      }
      // P_d of plane p = r - 2 (cell-centred)
      {
        const int p = r - 2;
        C P = C(0.f);
        if (pos && (FAST || (p >= 2 && p < sd - 2))) {
          const C uc = bg.V[d] + halve(vw[0] + vw[1]);
          const C Fc = halve(Fw[0] + Fw[1]);
          const C wsv = upwind_v(ww[d][0], ww[d][1], ww[d][2], ww[d][3], uc, uc * dtdx);
          P = bg.V[d] * Fc + wsv * (F0 + Fc);
        }
        Pd[0] = Pd[1];
        Pd[1] = P;
      }
      // conservative update of plane u = r - 2
      const int u = r - 2;
      if (owned && (FAST || (u >= m0 && u < m1))) {
        const int c = cxr + u * stM;
        C rv = rw[1], evv = er[0];
        if (FAST || (u >= 2 && u < sd - 2)) {
          C Flo = Fw[0], Fhi = Fw[1], Elo = Ew[0], Ehi = Ew[1];
          if (!FAST && L.has_child) {
            int g[3];
            gcoord(u, g);
            frontier_fluxes(L, d, g, Flo, Fhi, Elo, Ehi);
          }
          rv = rv - (Fhi - Flo) * iv;
          evv = evv - (Ehi - Elo) * iv;
        }
        st(rhoD, c, rv);
        st(eD, c, evv);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          C pv = pw[m][0];
          if (m == d) {
            if (FAST || (u >= 3 && u < sd - 2)) pv = pv - (Pd[1] - Pd[0]) * iv;
          } else {
            const int j = m == mx ? 0 : 1;
            if ((FAST || (u >= 2 && u < sd - 2)) && (j == 0 ? x >= 1 : row >= 1))
              pv = pv - (Pm[j][1] - Pm[j][0]) * iv;
          }
          st(piD[m], c, pv);
        }
      }
    };
    load(m0 - 3, nr, ne, nv, np);
    for (int i = 0; i < nit; ++i) {
      const int r = m0 - 3 + i;
      const bool fast = r >= r_lo && r <= r_hi &&
                        !(L.is_child && (r - 1 == L.G || r - 1 == L.G + L.n[d])) &&
                        !(L.has_child && near_frontier(L, d, r - 2));
      if (fast)
        step(i, std::true_type{});
      else
        step(i, std::false_type{});
    }
  } else {
    // ======================================================== x sweep, march in z
    C pr_r = C(0.f), pr_v = C(0.f), pr_F = C(0.f);  // plane r - 1 at (x, row)
    const int nit = m1 - m0 + 1;
    load(m0 - 1, nr, ne, nv, np);
    for (int i = 0; i < nit; ++i) {
      const int r = m0 - 1 + i;
      const C rc = nr, ec = ne, vc = nv, pi0 = np[0], pi1 = np[1], pi2 = np[2];
      if (i + 1 < nit) load(r + 1, nr, ne, nv, np);
      const C ep = eps_dev(ec, rc, bg);
      const C r_m2 = shfl_up(rc, 2), r_m1 = shfl_up(rc, 1), r_p1 = shfl_dn(rc, 1);
      const C e_m2 = shfl_up(ep, 2), e_m1 = shfl_up(ep, 1), e_p1 = shfl_dn(ep, 1);
      const bool pok = pos && (unsigned)r < (unsigned)sMU;
      // mass and energy flux at the x-face of this cell
      C Fv = C(0.f), Evv = C(0.f);
      if (pok && x >= 2 && x < sd - 1) {
        const C u = bg.V[0] + vc;
        const C cour = u * dtdx;
        const C drs = upwind_v(r_m2, r_m1, rc, r_p1, u, cour);
        Fv = (bg.rho0 * vc + drs * u) * Adt;
        const C des = upwind_v(e_m2, e_m1, ep, e_p1, u, cour);
        Evv = bg.eps0 * Fv + des * (F0 + Fv);
      }
      if (L.is_child && owned && r >= m0 && r < m1 && (x == L.G || x == L.G + L.n[0])) {
        // CommFlux record: transverse axes y (the row) and z (the march)
        fr_put(L, 0, x, row, r, 0, it.sub, as_double(Fv));
        fr_put(L, 0, x, row, r, 1, it.sub, as_double(Evv));
      }
      // rho, v_x, F of the row below
      C* xb = xch + (i & 1) * 3 * NT;
      xb[tid] = rc;
      xb[NT + tid] = vc;
      xb[2 * NT + tid] = Fv;
      __syncthreads();
      // plane m0 - 1 only feeds the z-fluxes of plane m0; the halo row only supplies
      // rho, v_x and F
      if (i > 0 && warp > 0) {
        const C r_rb = xb[tid - 32], v_rb = xb[NT + tid - 32], F_rb = xb[2 * NT + tid - 32];
        // w of this plane: along x (lane below), y (row below), z (previous plane)
        C wx = C(0.f), wy = C(0.f), wz = C(0.f);
        if (pok && x >= 1) {
          const C drf = halve(r_m1 + rc);
          wx = hdiv(pi0 - bg.V[0] * drf, bg.rho0 + drf);
        }
        if (pok && row >= 1) {
          const C drf = halve(r_rb + rc);
          wy = hdiv(pi1 - bg.V[1] * drf, bg.rho0 + drf);
        }
        if (pok && r >= 1) {
          const C drf = halve(pr_r + rc);
          wz = hdiv(pi2 - bg.V[2] * drf, bg.rho0 + drf);
        }
        const C wx_m1 = shfl_up(wx, 1), wx_p1 = shfl_dn(wx, 1), wx_p2 = shfl_dn(wx, 2);
        const C wy_m2 = shfl_up(wy, 2), wy_m1 = shfl_up(wy, 1), wy_p1 = shfl_dn(wy, 1);
        const C wz_m2 = shfl_up(wz, 2), wz_m1 = shfl_up(wz, 1), wz_p1 = shfl_dn(wz, 1);
        const C v_p1 = shfl_dn(vc, 1), F_p1 = shfl_dn(Fv, 1), E_p1 = shfl_dn(Evv, 1);
        // momentum fluxes: P_x cell-centred, P_y and P_z on the x-y and x-z edges
        C Px = C(0.f), Py = C(0.f), Pz = C(0.f);
        if (pok && x >= 2 && x < sd - 2) {
          const C uc = bg.V[0] + halve(vc + v_p1);
          const C Fc = halve(Fv + F_p1);
          const C wsv = upwind_v(wx_m1, wx, wx_p1, wx_p2, uc, uc * dtdx);
          Px = bg.V[0] * Fc + wsv * (F0 + Fc);
        }
        if (pok && x >= 2 && x < sd - 1 && row >= 1) {
          const C ue = bg.V[0] + halve(v_rb + vc);
          const C Fe = halve(F_rb + Fv);
          const C wsv = upwind_v(wy_m2, wy_m1, wy, wy_p1, ue, ue * dtdx);
          Py = bg.V[1] * Fe + wsv * (F0 + Fe);
        }
        if (pok && x >= 2 && x < sd - 1 && r >= 1) {
          const C ue = bg.V[0] + halve(pr_v + vc);
          const C Fe = halve(pr_F + Fv);
          const C wsv = upwind_v(wz_m2, wz_m1, wz, wz_p1, ue, ue * dtdx);
          Pz = bg.V[2] * Fe + wsv * (F0 + Fe);
        }
        const C Px_m1 = shfl_up(Px, 1), Py_p1 = shfl_dn(Py, 1), Pz_p1 = shfl_dn(Pz, 1);
        // conservative update of this cell
        if (owned && r >= m0 && r < m1) {
          const int c = cxr + r * stM;
          C rv = rc, evv = ec;
          if (x >= 2 && x < sd - 2) {
            C Flo = Fv, Fhi = F_p1, Elo = Evv, Ehi = E_p1;
            if (L.has_child) {
              int g[3];
              gcoord(r, g);
              frontier_fluxes(L, 0, g, Flo, Fhi, Elo, Ehi);
            }
            rv = rv - (Fhi - Flo) * iv;
            evv = evv - (Ehi - Elo) * iv;
          }
          st(rhoD, c, rv);
          st(eD, c, evv);
          C p0 = pi0, p1 = pi1, p2 = pi2;
          if (x >= 3 && x < sd - 2) p0 = p0 - (Px - Px_m1) * iv;
          if (x >= 2 && x < sd - 2 && row >= 1) p1 = p1 - (Py_p1 - Py) * iv;
          if (x >= 2 && x < sd - 2 && r >= 1) p2 = p2 - (Pz_p1 - Pz) * iv;
          st(piD[0], c, p0);
          st(piD[1], c, p1);
          st(piD[2], c, p2);
        }
      }
      pr_r = rc;
      pr_v = vc;
      pr_F = Fv;
    }
  }
}

// velocity from the transported momenta, then the second half kick S(dt/2); NC cells
// per thread as in el_source.  KICK2: the first sub-cycle of a finest level, whose
// second sub-cycle follows with nothing in between that changes the level: the
// second sub-cycle's first kick S(dt/2) is applied here too, as el_source computes it
// from the stored velocity (so with the same bits), and the momenta its transport
// starts from are written; that sub-cycle runs no kick of its own.
template <class T, int NC, int KICK2>
__device__ __forceinline__ void el_vrec_source(const LevelView& L, const Box& b, const Scratch& S,
                                               const Arith<T>* __restrict__ dtp, Arith<T> gm1,
                                               const Bg<Arith<T>>& bg, const Geo<Arith<T>>& g,
                                               int fused, int write_pi, const unsigned* el) {
  using C = Arith<T>;
  int c[NC], c3[NC][3];
  bool ok[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    int i, j, k;
    ok[n] = decode(b, el[n], i, j, k);
    if (NC == 1 && !ok[n]) return;
    if (!ok[n]) i = j = k = 1;
    c[n] = cidx(L, i, j, k);
    c3[n][0] = i;
    c3[n][1] = j;
    c3[n][2] = k;
  }
  St<T>* rhoA = (St<T>*)L.q[F_RHO];
  St<T>* eA = (St<T>*)L.q[F_E];
  // after fused sweeps the box's state is in Scratch::qb; outside the box it is in
  // the level's arrays, which this op then updates for the box
  const St<T>* rho = fused ? (const St<T>*)S.qb[0] : rhoA;
  const St<T>* e = fused ? (const St<T>*)S.qb[1] : eA;
  const Arith<T>* __restrict__ phi = (const Arith<T>*)L.phi;
  const C h = halve(dtp[0]);
  St<T> rc_s[NC], ec_s[NC];
  C rc[NC], ec[NC], fc[NC], rm[NC][3], em[NC][3], fm[NC][3], pv[NC][3];
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    rc_s[n] = rho[c[n]];
    ec_s[n] = e[c[n]];
    rc[n] = ld(rho, c[n]);
    ec[n] = ld(e, c[n]);
    fc[n] = ld(phi, c[n]);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (c3[n][d] >= 1) {
        const int m = c[n] - L.st[d];
        const bool own = !fused || c3[n][d] - 1 >= b.lo[d];
        rm[n][d] = ld(own ? rho : (const St<T>*)rhoA, m);
        em[n][d] = ld(own ? e : (const St<T>*)eA, m);
        fm[n][d] = ld(phi, m);
        pv[n][d] = ld((const C*)(fused ? S.qb[2 + d] : S.pi[d]), c[n]);
      }
  }
#pragma unroll
  for (int n = 0; n < NC; ++n) {
    if (!ok[n]) continue;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (c3[n][d] < 1) {
        if (KICK2 && write_pi) ((Arith<T>*)S.pi[d])[c[n]] = C(0.f);
        continue;
      }
      C drf = halve(rm[n][d] + rc[n]);
      C rinv = div_u(C(1.f), bg.rho0 + drf);
      C v = mul_u(sub_ky(pv[n][d], bg.V[d], drf), rinv);
      C acc = mul_u(mul_u(mul_u(gm1, ec[n] - em[n][d]), rinv) + (fc[n] - fm[n][d]),
                    g.inv_dx[d]);
      C vn = v - mul_u(h, acc);
      if (KICK2) {  // the same expression as the kick's
        const C rf = bg.rho0 + drf;
        const C acc2 = mul_u(div_u(mul_u(gm1, ec[n] - em[n][d]), rf) + (fc[n] - fm[n][d]),
                             g.inv_dx[d]);
        vn = as_stored(vn) - mul_u(h, acc2);
        if (write_pi)
          st((Arith<T>*)S.pi[d], c[n], mul_u(bg.rho0, vn) + mul_u(drf, add_k(vn, bg.V[d])));
      }
      st((St<T>*)L.q[F_VX + d], c[n], vn);
    }
    if (fused) {
      rhoA[c[n]] = rc_s[n];
      eA[c[n]] = ec_s[n];
    }
  }
}

// ------------------------------------------------------ level-0 boundaries
template <class T>
__device__ __forceinline__ void el_bc_axis(const LevelView& L, int d, int type_lo, int type_hi,
                                           T V0, T V1, T V2, unsigned tid) {
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  long long t = tid;
  const int G = L.G, n = L.n[d];
  long long per = (long long)L.s[t1] * L.s[t2];
  long long total = per * 2 * G * 5;
  if (t >= total) return;
  int f = (int)(t / (per * 2 * G));
  long long r = t - (long long)f * per * 2 * G;
  int side = (int)(r / (per * G));
  r -= (long long)side * per * G;
  int g = 1 + (int)(r / per);
  r -= (long long)(g - 1) * per;
  int b = (int)(r / L.s[t1]);
  int a = (int)(r - (long long)b * L.s[t1]);
  int type = side ? type_hi : type_lo;
  if (type < 0) return;  // this side is left alone (mirror fill of finer levels)
  int normal = (f == F_VX + d);
  int dst = side == 0 ? G - g : G + n - 1 + g, src = -1;
  T sign = T(1), fixed = T(0), shift = T(0);
  bool use_fixed = false;
  const T Vd = d == 0 ? V0 : (d == 1 ? V1 : V2);
  switch (type) {
    case 0:  // periodic
      src = side == 0 ? dst + n : dst - n;
      break;
    case 1:  // outflow: the nearest active element; for v_d the boundary face itself
             // (G or G + n), which the solver owns on both sides
      if (normal && side == 1) {
        if (g == 1) return;
        src = G + n;
      } else {
        src = side == 0 ? G : G + n - 1;
      }
      break;
    case 2:  // inflow: the background itself, zero deviation
      use_fixed = true;
      fixed = T(0);
      break;
    default:  // reflect
      if (!normal) {
        src = side == 0 ? G - 1 + g : G + n - g;
      } else {
        // v_ghost = -v_mirror, so dv_ghost = -dv_mirror - 2 V_d; wall face v = 0
        sign = T(-1);
        shift = T(-2) * Vd;
        if (side == 0) {
          src = G + g;
        } else {
          int gp = dst - (G + n);
          if (gp == 0) {
            use_fixed = true;
            fixed = -Vd;
          } else {
            src = G + n - gp;
          }
        }
      }
      break;
  }
  int c3[3];
  c3[t1] = a;
  c3[t2] = b;
  c3[d] = dst;
  St<T>* q = (St<T>*)L.q[f];
  int cd = (c3[2] * L.s[1] + c3[1]) * L.s[0] + c3[0];
  if (use_fixed) {
    put(q, cd, fixed);
  } else {
    c3[d] = src;
    int cs = (c3[2] * L.s[1] + c3[1]) * L.s[0] + c3[0];
    if (sign == T(1) && shift == T(0))
      q[cd] = q[cs];  // a copy keeps the stored value as it is
    else
      put(q, cd, sign * val(q, cs) + shift);
  }
  // the lower boundary face G of v_d: 0 at a wall, V (zero deviation) on an injection
  // face; the upper boundary face G + n is the g = 1 element of the upper side
  if ((type == 3 || type == 2) && side == 0 && normal && g == 1) {
    c3[d] = G;
    put(q, (c3[2] * L.s[1] + c3[1]) * L.s[0] + c3[0], type == 3 ? -Vd : T(0));
  }
}

// ---------------------------------------------------------------- CommUp
// A coarse host element holds 2 x 2 x 2 fine elements; CommUp fills the fine ghosts.
// Per field, the hosts with a ghost among their fine elements form the shell of
// their host box around the hosts whose fine elements are all kept (active cells;
// for v_d the faces strictly inside along d, so both frontier faces of v_d are
// filled).  The shell is cut into six disjoint boxes (two slabs across z over the
// whole x-y range, two across y, two across x), each into tiles of at most
// kCuHosts hosts in one host z-plane, one 256-thread chunk per tile.  The z pass
// interpolates each coarse column of a tile and its halo once (to both fine z
// offsets) into shared memory, the y pass each x-column once (to both fine y
// offsets), and the x pass gives a host's 8 fine elements: the arithmetic of
// interpolating each fine element alone along z, then y, then x, with every slope
// computed once per tile.  Along a staggered field's own axis the fine faces lie on
// the host face (copied) or midway to the next one (mean of the two, which favours
// neither side), so a mirror-symmetric coarse state gives mirror-symmetric ghosts.
static_assert(kCuHosts == kBlock, "one thread per host of a CommUp tile");

template <class T>
__device__ __forceinline__ void el_commup(const LevelView& C, const LevelView& F, unsigned tid) {
  using A = Arith<T>;  // the interpolation runs in the stencils' arithmetic type
  __shared__ A s_z[2][kCuZ];  // [fine z offset][column (y, x) of the tile and halo]
  __shared__ A s_y[4][kCuY];  // [fine z offset * 2 + fine y offset][(host y, x column)]
  __shared__ CuBox s_box;
  __shared__ int s_fr[2];     // field (-1: past the last tile) and tile within the box
  const int lt = (int)(tid % kBlock);
  // warp 0 finds the chunk's field and box: lane i takes box i % 6 of field i / 6
  if (lt < 32) {
    const int r = (int)(tid / kBlock);
    const int fb = lt < 30 ? lt : 29;
    const CuBox B = cu_box(F.n, F.G, fb / 6 >= F_VX ? fb / 6 - F_VX : -1, fb % 6);
    const int c = lt < 30 ? B.ez * B.ntx * B.nty : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lt >= o) incl += v;
    }
    const bool hit = r >= incl - c && r < incl;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      s_box = B;
      s_fr[0] = fb / 6;
      s_fr[1] = r - (incl - c);
    }
    if (lt == 0 && m == 0u) s_fr[0] = -1;
  }
  __syncthreads();
  const int f = s_fr[0];
  if (f < 0) return;  // uniform over the block
  const CuBox B = s_box;
  const int r = s_fr[1];
  const int sa = f >= F_VX ? f - F_VX : -1;
  const int per = B.ntx * B.nty;
  const int pz = r / per, rt = r - pz * per;
  const int tyi = rt / B.ntx, txi = rt - tyi * B.ntx;
  const int h2 = B.z0 + pz;
  const int X0 = B.x0 + txi * B.tx, Y0 = B.y0 + tyi * B.ty;
  const int wx = min(B.tx, B.x0 + B.ex - X0), wy = min(B.ty, B.y0 + B.ey - Y0);
  const int P = wx + 2;  // pitch of a row of columns
  // the two centred fine positions lie at -1/4 and +1/4 of a coarse cell: q0 -+ half
  // of the half slope hslope returns
  const St<T>* q = (const St<T>*)C.q[f];
  // z pass: the tile's columns and a halo of one (hosts in [-G/2 - 1, n/2 + G/2])
  for (int e = lt; e < P * (wy + 2); e += kBlock) {
    const int cy = e / P, cx = e - cy * P;
    const int hx = X0 - 1 + cx, hy = Y0 - 1 + cy;
    const int k = ((C.G + F.off[2] + h2) * C.s[1] + C.G + F.off[1] + hy) * C.s[0] + C.G +
                  F.off[0] + hx;
    const A qm = ld(q, k - C.st[2]), q0 = ld(q, k), qp = ld(q, k + C.st[2]);
    if (sa == 2) {
      s_z[0][e] = q0;
      s_z[1][e] = halve(q0 + qp);
    } else {
      const A sl = hslope(q0 - qm, qp - q0);
      s_z[0][e] = q0 - halve(sl);
      s_z[1][e] = q0 + halve(sl);
    }
  }
  __syncthreads();
  // y pass: every x column of the tile's host rows
  for (int e = lt; e < 2 * wy * P; e += kBlock) {
    const int iz = e / (wy * P), rem = e - iz * wy * P;
    const A qm = s_z[iz][rem], q0 = s_z[iz][rem + P], qp = s_z[iz][rem + 2 * P];
    if (sa == 1) {
      s_y[2 * iz][rem] = q0;
      s_y[2 * iz + 1][rem] = halve(q0 + qp);
    } else {
      const A sl = hslope(q0 - qm, qp - q0);
      s_y[2 * iz][rem] = q0 - halve(sl);
      s_y[2 * iz + 1][rem] = q0 + halve(sl);
    }
  }
  __syncthreads();
  // x pass and stores: one host per thread
  if (lt >= wx * wy) return;
  const int ty = lt / wx, tx = lt - ty * wx;
  const int h0 = X0 + tx, h1 = Y0 + ty;
  St<T>* out = (St<T>*)F.q[f];
  const int G = F.G;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int iz = j >> 1, iy = j & 1;
    const A* row = s_y[j] + ty * P + tx;
    const A qm = row[0], q0 = row[1], qp = row[2];
    A v[2];
    if (sa == 0) {
      v[0] = q0;
      v[1] = halve(q0 + qp);
    } else {
      const A sl = hslope(q0 - qm, qp - q0);
      v[0] = q0 - halve(sl);
      v[1] = q0 + halve(sl);
    }
    // the two fine elements along x are neighbours in memory: one vector store when
    // both are ghosts and the pair starts on an even element (aligned)
    const int fi0 = G + 2 * h0, fj = G + 2 * h1 + iy, fk = G + 2 * h2 + iz;
    const bool yz = fj >= G + (sa == 1) && fj < G + F.n[1] && fk >= G + (sa == 2) &&
                    fk < G + F.n[2];
    const bool act0 = yz && fi0 >= G + (sa == 0) && fi0 < G + F.n[0];
    const bool act1 = yz && fi0 + 1 >= G + (sa == 0) && fi0 + 1 < G + F.n[0];
    const int e0 = (fk * F.s[1] + fj) * F.s[0] + fi0;
    if (!act0 && !act1 && (e0 & 1) == 0) {
      st2(out, e0, v[0], v[1]);
      continue;
    }
#pragma unroll
    for (int ix = 0; ix < 2; ++ix) {
      const bool act = ix == 0 ? act0 : act1;
      if (!act) st(out, e0 + ix, v[ix]);
    }
  }
}

// -------------------------------------------------------------- CommMean
__device__ __forceinline__ bool in_band(const LevelView& F, int band, int a0, int a1, int a2) {
  int a3[3] = {a0, a1, a2};
  int dist = 1 << 30;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int lo = a3[d] - F.off[d], hi = F.off[d] + (F.n[d] >> 1) - 1 - a3[d];
    if (lo < 0 || hi < 0) return false;
    if (F.mir >> d & 1) lo = 1 << 30;  // a mirror face bounds no band
    dist = min(dist, min(lo, hi));
  }
  return dist < band;
}

template <class T>
__device__ __forceinline__ void el_commmean(const LevelView& C, const LevelView& F, int band, unsigned tid) {
  const unsigned t = tid;  // coarse cells of the covered box: fewer than 2^31
  const unsigned h0 = F.n[0] >> 1, h1 = F.n[1] >> 1, h2 = F.n[2] >> 1;
  if (t >= h0 * h1 * h2) return;
  const unsigned q = t / h0;
  int a = (int)(t - q * h0), b = (int)(q % h1), cc = (int)(q / h1);
  int r[3] = {a, b, cc};
  int a3[3] = {a + F.off[0], b + F.off[1], cc + F.off[2]};
  const int Gf = F.G, Gc = C.G;
  int dst = ((Gc + a3[2]) * C.s[1] + Gc + a3[1]) * C.s[0] + Gc + a3[0];
  if (in_band(F, band, a3[0], a3[1], a3[2])) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const St<T>* q = (const St<T>*)F.q[f];
      Arith<T> sz[2];
#pragma unroll
      for (int dz = 0; dz < 2; ++dz) {
        Arith<T> sy[2];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
          int c0 = ((Gf + 2 * cc + dz) * F.s[1] + Gf + 2 * b + dy) * F.s[0] + Gf + 2 * a;
          sy[dy] = ld(q, c0) + ld(q, c0 + 1);
        }
        sz[dz] = sy[0] + sy[1];
      }
      st((St<T>*)C.q[f], dst, pow2_times(sz[0] + sz[1], 0.125f));
    }
  }
#pragma unroll
  for (int sa = 0; sa < 3; ++sa) {
    if (r[sa] == 0) continue;
    int m3[3] = {a3[0], a3[1], a3[2]};
    m3[sa] -= 1;
    if (!in_band(F, band, a3[0], a3[1], a3[2]) && !in_band(F, band, m3[0], m3[1], m3[2])) continue;
    int t1 = sa == 0 ? 1 : 0, t2 = sa == 2 ? 1 : 2;
    const St<T>* q = (const St<T>*)F.q[F_VX + sa];
    Arith<T> sv[2];
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      Arith<T> pair[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        int fi[3];
        fi[sa] = Gf + 2 * r[sa];
        fi[t1] = Gf + 2 * r[t1] + u;
        fi[t2] = Gf + 2 * r[t2] + v;
        pair[u] = ld(q, (fi[2] * F.s[1] + fi[1]) * F.s[0] + fi[0]);
      }
      sv[v] = pair[0] + pair[1];
    }
    st((St<T>*)C.q[F_VX + sa], dst, pow2_times(sv[0] + sv[1], 0.25f));
  }
}

// ------------------------------------------------------------- time step
__device__ __forceinline__ float warp_max_t(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// the larger of two double-float values (a total order on normalised pairs: hi, then
// lo); a NaN operand loses, as in fmax
__device__ __forceinline__ df64 dmax(df64 a, df64 b) {
  return (a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo) || b.hi != b.hi) ? a : b;
}
__device__ __forceinline__ df64 warp_max_t(df64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = dmax(v, df64(__shfl_xor_sync(0xffffffffu, v.hi, o),
                     __shfl_xor_sync(0xffffffffu, v.lo, o)));
  return v;
}
__device__ __forceinline__ df64 dabs(df64 v) { return v.hi < 0.f ? -v : v; }
// Square root in double-float: the float root s refined by one Newton step on the
// square (Heron's method; the double-length form of Karp & Markstein, ACM TOMS 23,
// 1997): s + (x - s^2) / (2 s), with s^2 exact as a product plus its error, so the
// residual is exact up to the low parts and the result good to about 2^-46.  For
// x <= 0 (an unhealthy state, flagged by the caller) the float root of hi.
__device__ __forceinline__ df64 dsqrt(df64 x) {
  const float s = sqrtf(x.hi);
  if (!(x.hi > 0.f)) return df64(s);
  const df64 s2 = two_prod(s, s);
  const float r = ((x.hi - s2.hi) - s2.lo + x.lo) * (0.5f * rcp_est(s));
  return fast_two_sum(s, r);
}

// Per-level Courant limit: min over active cells and axes of cfl dx_d / (cs + |v_d|).
// Division is correctly rounded and monotone, so that minimum equals
// cfl dx_d / max(cs + |v_d|): the kernel reduces the per-axis maxima (one division
// per level instead of three per cell); a maximum is exact in any precision, so it
// is taken in the per-cell type and widened once per block.  Per-cell arithmetic:
// FP32 for the FP32 state (FP32 sound speeds); double-float for the FP64 state (its
// sound speed and |v| within about 2^-44, so the limit is within that of the FP64
// one; the FP64 pipe would take ~40 operations per cell).  The maxima, the minimum
// over levels and dt itself are FP64.  Also flags NaN, rho <= 0 or e <= 0.
constexpr int kDtCells = 4;
template <class T>
__device__ __forceinline__ void el_dt_level(const LevelView& L, const Box& b, int level, double gg,
                                            Arith<T> gga, int hydro, DevScalars* ds,
                                            double rho0, double e0, double V0, double V1,
                                            double V2, const Bg<Arith<T>>& bg,
                                            unsigned tid) {
  using A = Arith<T>;
  __shared__ A sm[3][kBlock / 32];
  __shared__ int bad_s;
  if (threadIdx.x == 0) bad_s = 0;
  __syncthreads();
  A mx[3] = {A(0.f), A(0.f), A(0.f)};
  // kDtCells cells per thread (strided by the block size), every load first: a block
  // then issues one atomic per axis for kBlock kDtCells cells
  int cc[kDtCells];
  bool in[kDtCells];
#pragma unroll
  for (int u = 0; u < kDtCells; ++u) {
    const unsigned t = (tid / kBlock) * kBlock * kDtCells + u * kBlock + threadIdx.x;
    int i, j, k;  // b is the active box: multiply-shift division, no 64-bit divide
    in[u] = decode(b, t, i, j, k);
    cc[u] = in[u] ? (k * L.s[1] + j) * L.s[0] + i : (L.G * L.s[1] + L.G) * L.s[0] + L.G;
  }
  const St<T>* v3[3] = {(const St<T>*)L.q[F_VX], (const St<T>*)L.q[F_VX + 1],
                        (const St<T>*)L.q[F_VX + 2]};
  bool bad = false;
  if constexpr (sizeof(T) == 4) {
    float rho[kDtCells], e[kDtCells], va[kDtCells][3], vb[kDtCells][3];
#pragma unroll
    for (int u = 0; u < kDtCells; ++u) {
      const int c = cc[u];
      rho[u] = val((const St<T>*)L.q[F_RHO], c);
      e[u] = val((const St<T>*)L.q[F_E], c);
      if (hydro)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          va[u][d] = val(v3[d], c);
          vb[u][d] = val(v3[d], c + L.st[d]);
        }
    }
    const float Vb[3] = {(float)V0, (float)V1, (float)V2};
#pragma unroll
    for (int u = 0; u < kDtCells; ++u) {
      if (!in[u]) continue;
      const float r = (float)rho0 + rho[u], ee = (float)e0 + e[u];
      if (!(r > 0.f) || !(ee > 0.f)) bad = true;
      if (hydro) {
        const float cs = sqrtf((float)gg * ee / r);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const float v0 = fabsf(Vb[d] + va[u][d]), v1 = fabsf(Vb[d] + vb[u][d]);
          const float m = cs + (v0 > v1 ? v0 : v1);
          mx[d] = m > mx[d] ? m : mx[d];
        }
      }
    }
  } else {
    A rho[kDtCells], e[kDtCells], va[kDtCells][3], vb[kDtCells][3];
#pragma unroll
    for (int u = 0; u < kDtCells; ++u) {
      const int c = cc[u];
      rho[u] = ld((const St<T>*)L.q[F_RHO], c);
      e[u] = ld((const St<T>*)L.q[F_E], c);
      if (hydro)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          va[u][d] = ld(v3[d], c);
          vb[u][d] = ld(v3[d], c + L.st[d]);
        }
    }
#pragma unroll
    for (int u = 0; u < kDtCells; ++u) {
      if (!in[u]) continue;
      const A r = bg.rho0 + rho[u], ee = bg.e0 + e[u];
      if (!gt0(r) || !gt0(ee)) bad = true;
      if (hydro) {
        const A cs = dsqrt(hdiv(gga * ee, r));
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const A v0 = dabs(bg.V[d] + va[u][d]), v1 = dabs(bg.V[d] + vb[u][d]);
          mx[d] = dmax(mx[d], cs + dmax(v0, v1));
        }
      }
    }
  }
  if (bad) bad_s = 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    A v = warp_max_t(mx[d]);
    if ((threadIdx.x & 31) == 0) sm[d][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      A v = threadIdx.x < kBlock / 32 ? sm[d][threadIdx.x] : A(0.f);
      v = warp_max_t(v);
      // non-negative doubles order like their bit patterns (NaN is caught above)
      const double w = as_double(v);
      if (threadIdx.x == 0 && w > 0.0)
        atomicMax(&ds->dtmin[3 * level + d], (unsigned long long)__double_as_longlong(w));
    }
    if (threadIdx.x == 0 && bad_s) atomicOr(&ds->unhealthy, 1);
  }
}

// Eq. 55: dt = min_l dt_l prod_{m<l} xi_m; resets the per-level maxima
__device__ __forceinline__ void el_dt_finalize(DevScalars* ds, int n_levels, const DtFinal& fin,
                                               double dt_fixed) {
  __shared__ double s_lim[16];
  __shared__ double s_ratio[kBlock];
  __shared__ int s_word[kBlock];
  if (threadIdx.x == 0) {
    for (int l = 0; l < n_levels; ++l) {
      double lim = fin.diff_lim[l];
      for (int d = 0; d < 3; ++d) {
        double mx = __longlong_as_double((long long)ds->dtmin[3 * l + d]);
        double t = fin.cfl_dx[l][d] / mx;  // +inf when the maximum is 0
        if (t < lim) lim = t;
        ds->dtmin[3 * l + d] = 0ull;
      }
      ds->dtlev[l] = lim;
      s_lim[l] = lim;
    }
  }
  __syncthreads();
  double prod[16];
  unsigned xi1 = 0;
  if (fin.search && n_levels > 1) {
    // Eq. 55-56: the word xi_m in {1, 2} (bit m of w set: xi_m = 2) with the largest
    // step per unit cost; ties go to the smallest w, as a sequential scan keeps the
    // first maximum
    const int nw = n_levels - 1;
    double best = -1.0;
    int bw = 0;
    for (int w = threadIdx.x; w < (1 << nw); w += kBlock) {
      double dt = INFINITY, C = 0.0, pr = 1.0;
      for (int l = 0; l < n_levels; ++l) {
        if (l > 0) pr *= ((w >> (l - 1)) & 1) ? 2.0 : 1.0;
        const double t = s_lim[l] * pr;
        if (t < dt) dt = t;
        C += fin.cost[l] * pr;
      }
      const double ratio = dt / C;
      if (ratio > best) {
        best = ratio;
        bw = w;
      }
    }
    s_ratio[threadIdx.x] = best;
    s_word[threadIdx.x] = bw;
    __syncthreads();
    for (int h = kBlock / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) {
        const double r2 = s_ratio[threadIdx.x + h];
        const int w2 = s_word[threadIdx.x + h];
        if (r2 > s_ratio[threadIdx.x] || (r2 == s_ratio[threadIdx.x] && w2 < s_word[threadIdx.x])) {
          s_ratio[threadIdx.x] = r2;
          s_word[threadIdx.x] = w2;
        }
      }
      __syncthreads();
    }
    const int w = s_word[0];
    double pr = 1.0;
    for (int l = 0; l < n_levels; ++l) {
      if (l > 0) {
        const bool two = (w >> (l - 1)) & 1;
        pr *= two ? 2.0 : 1.0;
        if (!two) xi1 |= 1u << (l - 1);
      }
      prod[l] = pr;
    }
  } else {
    for (int l = 0; l < n_levels; ++l) prod[l] = fin.prod[l];
  }
  if (threadIdx.x != 0) return;
  double dt = INFINITY;
  for (int l = 0; l < n_levels; ++l) {
    double t = s_lim[l] * prod[l];
    if (t < dt) dt = t;
  }
  if (dt_fixed > 0.0) dt = dt_fixed;
  ds->dt = dt;
  ds->xi1 = xi1;
  // level steps take dt / prod_{m<l} xi_m (a power of two: exact)
  for (int l = 0; l < n_levels; ++l) {
    double dl = dt / prod[l];
    ds->dtl[l] = dl;
    ds->dtf[l] = (float)dl;
    ds->dtd[l] = to_df64(dl);
    // the level step's constants, once here instead of in every thread
    for (int q = 0; q < 12; ++q) {
      const double k = fin.kfac[l][q] * dl;
      ds->kd[l][q] = to_df64(k);
      ds->kf[l][q] = (float)k;
    }
  }
}

__device__ __forceinline__ void el_time_advance(DevScalars* ds) {
  if (threadIdx.x == 0) ds->t += ds->dt;
}

// ------------------------------------------------------------------ force
// Eq. 18 on one level: F += (rho - rho0) w_c over uncovered active cells, with the
// static FP64 weight vectors w_c = GM V_c r_c / (r^2 + eps^2)^(3/2) precomputed
// (x, y and z components in three planes of fw).  Each thread accumulates
// kForceCells cells (strided by the block size) in FP64, then a fixed warp-shuffle
// tree and the 8 warp sums give one partial per block.
constexpr int kForceCells = 8;

template <class T>
__device__ __forceinline__ void el_force_level(const LevelView& L, const Box& b,
                                               const double* __restrict__ fw,
                                               double* partials, unsigned tid) {
  __shared__ double sw[3][kBlock / 32];
  const long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  const double* fx = fw;
  const double* fy = fw + na;
  const double* fz = fw + 2 * na;
  double f[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int u = 0; u < kForceCells; ++u) {
    const unsigned t = (tid / kBlock) * kBlock * kForceCells + u * kBlock + threadIdx.x;
    int i, j, k;  // b is the active box: multiply-shift division, no 64-bit divide
    if (!decode(b, t, i, j, k)) break;
    const int ai = i - L.G, aj = j - L.G, ak = k - L.G;
    bool covered = L.has_child && ai >= L.coff[0] && ai < L.coff[0] + (L.cn[0] >> 1) &&
                   aj >= L.coff[1] && aj < L.coff[1] + (L.cn[1] >> 1) && ak >= L.coff[2] &&
                   ak < L.coff[2] + (L.cn[2] >> 1);
    if (covered) continue;
    double dr = (double)val((const St<T>*)L.q[F_RHO], ((L.G + ak) * L.s[1] + L.G + aj) * L.s[0] + L.G + ai);
    f[0] += dr * fx[t];
    f[1] += dr * fy[t];
    f[2] += dr * fz[t];
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f[d] += __shfl_down_sync(0xffffffffu, f[d], o);
    if ((threadIdx.x & 31) == 0) sw[d][threadIdx.x >> 5] = f[d];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kBlock / 32; ++w) s += sw[threadIdx.x][w];
    partials[3 * (tid / kBlock) + threadIdx.x] = s;
  }
}

// static force weights of the active cells; with mirror planes the force is that of
// the unfolded domain: no component along a mirror axis, the others mult times the
// sum over the simulated part (mult = 2^planes scales exactly)
__global__ void __launch_bounds__(kBlock) k_force_weights(LevelView L, double GM, double eps,
                                                          double mult, double* fw) {
  long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  if (t >= na) return;
  int ai = (int)(t % L.n[0]);
  int aj = (int)((t / L.n[0]) % L.n[1]);
  int ak = (int)(t / ((long long)L.n[0] * L.n[1]));
  double x = L.lo[0] + (ai + 0.5) * L.dx[0];
  double y = L.lo[1] + (aj + 0.5) * L.dx[1];
  double z = L.lo[2] + (ak + 0.5) * L.dx[2];
  double r2 = x * x + y * y + z * z + eps * eps;
  double w = GM * L.vol / (r2 * sqrt(r2));
  fw[t] = L.mir & 1 ? 0.0 : mult * (w * x);
  fw[t + na] = L.mir & 2 ? 0.0 : mult * (w * y);
  fw[t + 2 * na] = L.mir & 4 ? 0.0 : mult * (w * z);
}

// fixed-order compensated (Neumaier) sum of the block partials, one warp per
// component (threads 96.. of the block only take part in the barrier)
__device__ __forceinline__ void el_force_finalize(const double* __restrict__ partials, int n,
                                                  DevScalars* ds, double* ring, int ring_cap,
                                                  long long* ring_pos) {
  int comp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (comp < 3) {
    double s = 0.0, cmp = 0.0;
    for (int p = lane; p < n; p += 32) {
      double v = partials[3 * p + comp];
      double tt = s + v;
      if (fabs(s) >= fabs(v))
        cmp += (s - tt) + v;
      else
        cmp += (v - tt) + s;
      s = tt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double so = __shfl_down_sync(0xffffffffu, s, o);
      double co = __shfl_down_sync(0xffffffffu, cmp, o);
      if (lane < o) {
        double tt = s + so;
        if (fabs(s) >= fabs(so))
          cmp += (s - tt) + so;
        else
          cmp += (so - tt) + s;
        s = tt;
        cmp += co;
      }
    }
    if (lane == 0) {
      double F = s + cmp;
      ds->F[comp] = F;
      if (ring) ring[kRingStride * (*ring_pos % ring_cap) + comp] = F;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && ring) {
    // the time at the end of this coarse step (the time update follows this op)
    ring[kRingStride * (*ring_pos % ring_cap) + 3] = ds->t + ds->dt;
    *ring_pos += 1;
  }
}

// ----------------------------------------------------------- initialisation
template <class T>
__global__ void __launch_bounds__(kBlock) k_init_uniform(LevelView L, T rho0, T e0, T V0, T V1,
                                                         T V2) {
  long long c = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (c >= L.nc) return;
  (void)rho0;
  (void)e0;
  (void)V0;
  (void)V1;
  (void)V2;
#pragma unroll
  for (int f = 0; f < 5; ++f) put((St<T>*)L.q[f], c, T(0));
}

// Plummer potential (Eq. 16, attractive sign) at every cell centre; luminosity
// weights on active cells and on their mirror images in the ghost layers (Gaussian
// weights are normalised afterwards)
template <class T>
__global__ void __launch_bounds__(kBlock) k_static(LevelView L, double GM, double eps,
                                                   double sigma, int vertex_ok, int vx0, int vx1,
                                                   int vx2) {
  long long c = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (c >= L.nc) return;
  int i = (int)(c % L.s[0]), j = (int)((c / L.s[0]) % L.s[1]),
      k = (int)(c / ((long long)L.s[0] * L.s[1]));
  double x = L.lo[0] + (i - L.G + 0.5) * L.dx[0];
  double y = L.lo[1] + (j - L.G + 0.5) * L.dx[1];
  double z = L.lo[2] + (k - L.G + 0.5) * L.dx[2];
  // the static fields are held in the stencils' arithmetic type (double-float for the
  // FP64 state): only the stencils read them
  ((Arith<T>*)L.phi)[c] = from_double<Arith<T>>(-GM / sqrt(x * x + y * y + z * z + eps * eps));
  bool act = i >= (L.mir & 1 ? 0 : L.G) && i < L.G + L.n[0] &&
             j >= (L.mir & 2 ? 0 : L.G) && j < L.G + L.n[1] &&
             k >= (L.mir & 4 ? 0 : L.G) && k < L.G + L.n[2];
  double lw = 0.0;
  if (act) {
    if (sigma > 0.0) {
      lw = exp(-(x * x + y * y + z * z) / (2.0 * sigma * sigma));
    } else if (vertex_ok) {
      int ai = i - L.G, aj = j - L.G, ak = k - L.G;
      if ((ai == vx0 - 1 || ai == vx0) && (aj == vx1 - 1 || aj == vx1) &&
          (ak == vx2 - 1 || ak == vx2))
        lw = 1.0 / (8.0 * L.vol);
    }
  }
  ((Arith<T>*)L.lumw)[c] = from_double<Arith<T>>(lw);
}

// Gaussian weights: fixed-order sum over the active cells (block tree, then one
// block in index order), so every context normalises to the same bits
template <class T>
__global__ void __launch_bounds__(kBlock) k_lum_partials(LevelView L, double* partials) {
  __shared__ double sm[kBlock];
  long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  double w = 0.0;
  if (t < na) {
    int i = (int)(t % L.n[0]), j = (int)((t / L.n[0]) % L.n[1]),
        k = (int)(t / ((long long)L.n[0] * L.n[1]));
    w = as_double(((const Arith<T>*)L.lumw)[((k + L.G) * L.s[1] + j + L.G) * L.s[0] + i + L.G]);
  }
  sm[threadIdx.x] = w;
  __syncthreads();
  for (int s = kBlock / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sm[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out) {
  __shared__ double sm[kBlock];
  double s = 0.0;
  for (int p = threadIdx.x; p < n; p += kBlock) s += partials[p];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_normalise_lum(LevelView L, const double* wsum,
                                                          double mult) {
  long long c = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (c >= L.nc) return;
  Arith<T>* lw = (Arith<T>*)L.lumw;
  // the unfolded domain holds mult copies of the active cells
  lw[c] = from_double<Arith<T>>(as_double(lw[c]) / (mult * wsum[0] * L.vol));
}

// host I/O: full values = background + stored deviation (bgv = 0 for raw state)
template <class T>
__global__ void __launch_bounds__(kBlock) k_pack(LevelView L, int field, double* out, int full,
                                                 double bgv) {
  long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
  const St<T>* q = (const St<T>*)L.q[field];
  if (full) {
    if (t < L.nc) out[t] = bgv + (double)val(q, t);
    return;
  }
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  if (t >= na) return;
  int i = (int)(t % L.n[0]), j = (int)((t / L.n[0]) % L.n[1]),
      k = (int)(t / ((long long)L.n[0] * L.n[1]));
  out[t] = bgv + (double)val(q, ((k + L.G) * L.s[1] + j + L.G) * L.s[0] + i + L.G);
}

template <class T>
__global__ void __launch_bounds__(kBlock) k_unpack(LevelView L, int field, const double* in,
                                                   int full, double bgv) {
  long long t = blockIdx.x * (long long)kBlock + threadIdx.x;
  St<T>* q = (St<T>*)L.q[field];
  if (full) {
    if (t < L.nc) put(q, t, (T)(in[t] - bgv));
    return;
  }
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  if (t >= na) return;
  int i = (int)(t % L.n[0]), j = (int)((t / L.n[0]) % L.n[1]),
      k = (int)(t / ((long long)L.n[0] * L.n[1]));
  put(q, ((k + L.G) * L.s[1] + j + L.G) * L.s[0] + i + L.G, (T)(in[t] - bgv));
}

// hdiv versus IEEE division on the given operands: max |error| in ulps of the IEEE
// quotient (as a double), over n pairs
__global__ void k_hdiv_check(const double* a, const double* b, int n, double* max_ulp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double u = 0.0;
  if (t < n) {
    double q = a[t] / b[t];
    double h = hdiv(a[t], b[t]);
    double aq = fabs(q);
    double ulp = __longlong_as_double(__double_as_longlong(aq) + 1) - aq;
    u = q == h ? 0.0 : fabs(h - q) / ulp;
  }
  for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
  if ((threadIdx.x & 31) == 0 && u > 0.0)
    atomicMax((unsigned long long*)max_ulp, (unsigned long long)__double_as_longlong(u));
}

// FP64 throughput probe: every thread runs kProbeChains independent chains of
// dependent fused multiply-adds (2 flops each); with a full SM of threads the FP64
// pipe, not the chain latency, sets the rate.  The result is written only when it
// takes an impossible value, so the work cannot be dropped and nothing is stored.
constexpr int kProbeChains = 8;
__global__ void __launch_bounds__(kBlock) k_dfma_probe(int iters, double* sink) {
  double a[kProbeChains];
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) a[i] = 1.0 + 1e-3 * (threadIdx.x + i);
  const double b = 0.999999999, c = 1e-9;
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = fma(a[i], b, c);
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kProbeChains; ++i) s += a[i];
  if (s == -1.0) sink[0] = s;
}

// double-float arithmetic on the device versus FP64 on n operand pairs: the largest
// error of conversion, sum, product and quotient, each in units of its bound
// (2^-45 |a|; 2^-46 (|a| + |b|); 2^-46 |a b| + 2^-120; 2^-42 |a / b| + 2^-120)
constexpr int kDf64Checks = 8;  // entries of df_check_df64's worst[]
__global__ void k_df64_check(const double* a, const double* b, int n, double* worst) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  double w[kDf64Checks] = {};
  if (t < n) {
    const df64 x = to_df64(a[t]), y = to_df64(b[t]);
    const double A = to_double(x), B = to_double(y);
    w[0] = fabs(A - a[t]) / (0x1.0p-45 * fabs(a[t]) + 1e-300);
    w[1] = fabs(to_double(x + y) - (A + B)) / (0x1.0p-46 * (fabs(A) + fabs(B)) + 1e-300);
    w[2] = fabs(to_double(x * y) - A * B) / (0x1.0p-46 * fabs(A * B) + 0x1.0p-120);
    w[3] = fabs(to_double(x / y) - A / B) / (0x1.0p-42 * fabs(A / B) + 0x1.0p-120);
    // the unnormalised product and quotient: their values (hi + lo in FP64) within
    // the same bounds, lo within 2^-21 of hi, and as an operand of the next sum
    const df64 mu = mul_u(x, y), qu = div_u(x, y);
    const double AB = A * B, Q = A / B;
    w[4] = fabs((double)mu.hi + (double)mu.lo - AB) / (0x1.0p-46 * fabs(AB) + 0x1.0p-120);
    w[5] = fabs((double)qu.hi + (double)qu.lo - Q) / (0x1.0p-42 * fabs(Q) + 0x1.0p-120);
    if (mu.hi != 0.f) w[6] = fabs((double)mu.lo) / (0x1.0p-21 * fabs((double)mu.hi));
    if (qu.hi != 0.f) w[6] = fmax(w[6], fabs((double)qu.lo) / (0x1.0p-21 * fabs((double)qu.hi)));
    if (fabs(AB) >= 0x1.0p-100)
      w[7] = fabs(to_double(mu + x) - (AB + A)) /
             (0x1.0p-45 * (fabs(AB) + fabs(A)) + 0x1.0p-120);
  }
  for (int q = 0; q < kDf64Checks; ++q) {
    double u = w[q];
    for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
    if ((threadIdx.x & 31) == 0 && u > 0.0)
      atomicMax((unsigned long long*)&worst[q], (unsigned long long)__double_as_longlong(u));
  }
}

}  // namespace

int launch_df64_check(const double* a, const double* b, int n, double* worst, cudaStream_t st) {
  k_df64_check<<<(n + 255) / 256, 256, 0, st>>>(a, b, n, worst);
  return 1;
}

long long launch_dfma_probe(int blocks, int iters, double* sink, cudaStream_t st) {
  k_dfma_probe<<<blocks, kBlock, 0, st>>>(iters, sink);
  return 2LL * kProbeChains * iters * (long long)kBlock * blocks;
}

int launch_hdiv_check(const double* a, const double* b, int n, double* max_ulp, cudaStream_t st) {
  k_hdiv_check<<<(n + 255) / 256, 256, 0, st>>>(a, b, n, max_ulp);
  return 1;
}

// =================================================================== work lists

// One op on one work item: maps the item's fields onto the element function.
// items inside a second sub-cycle that the Eq. 55-56 search dropped do nothing
template <class T>
__device__ __forceinline__ bool skipped(const Item<T>& it) {
  return it.br != 0u && (it.br & it.ds->xi1) != 0u;
}

template <class T, int OP, int D>
__device__ __forceinline__ void run_op(const Item<T>& it, unsigned tid) {
  if (skipped(it)) return;
  // elements of this thread: tid, or for the two-cell ops the same lane of both
  // halves of its 512-element chunk
  constexpr int NC = cells_per_thread(OP, (int)sizeof(T));
  unsigned el[NC];
  el[0] = NC == 1 ? tid : (tid / kBlock) * (NC * kBlock) + tid % kBlock;
#pragma unroll
  for (int n = 1; n < NC; ++n) el[n] = el[0] + n * kBlock;
  if (OP == OP_SOURCE)
    el_source<T, NC>(it.L, it.b, it.S, (const Arith<T>*)it.dt, it.flags & FL_WRITE_PI, it.gm1,
                     it.bg, it.g, el);
  else if (OP == OP_COMPRESS) {
    if (it.L.has_child)  // before any consumer
#pragma unroll 1
      for (int n = 0; n < NC; ++n) fr_sums(it.L, it.ds, it.level, el[n]);
    el_compress_lum<T, NC>(it.L, it.b, it.S, (const Arith<T>*)it.dt, it.gm1, it.lum,
                           it.flags & FL_SS3, it.flags & FL_LUM, it.flags & FL_EPS, it.bg, it.g,
                           el);
  }
  else if (OP == OP_FRONTIER_DIFF)
    el_frontier_diff<T>(it.L, it.S, (const Arith<T>*)it.kc, it.bg.rho0, it.flags & FL_DFR, it.sub,
                        tid);
  else if (OP == OP_DIFFUSE)  // D = 1: with the x sweep's preparation
    el_diffuse<T, NC, D>(it.L, it.b, it.S, (const Arith<T>*)it.kc, it.bg.rho0, it.flags & FL_DFR,
                         it.g, it.bg, el);
  else if (OP == OP_TPREP)
    el_tprep<T>(it.L, it.b, it.S, it.bg, it.flags & FL_EPS_ONLY, tid);
  else if (OP == OP_TFLUX)
    el_tflux<T, D>(it.L, it.b, it.S, (const Arith<T>*)it.kc, it.bg, it.sub, tid);
  else if (OP == OP_TMOM)
    el_tmom<T, D>(it.L, it.b, it.S, (const Arith<T>*)it.kc, it.bg, tid);
  else if (OP == OP_TUPDATE)
    el_tupdate<T, D, NC>(it.L, it.b, it.S, it.g, el);
  else if (OP == OP_VISC_Q)
    el_visc_q<T>(it.L, it.b, it.S, (const Arith<T>*)it.dt, it.av, it.bg, it.g, tid);
  else if (OP == OP_VISC_V)
    el_visc_v<T>(it.L, it.b, it.S, (const Arith<T>*)it.dt, it.flags & FL_WRITE_PI, it.bg, it.g, tid);
  else if (OP == OP_VREC)  // D = 1: with the next sub-cycle's first kick
    el_vrec_source<T, NC, D>(it.L, it.b, it.S, (const Arith<T>*)it.dt, it.gm1, it.bg, it.g,
                             it.flags & FL_FUSED, it.flags & FL_WRITE_PI, el);
  else if (OP == OP_BC)
    el_bc_axis<T>(it.L, D, it.bc_lo, it.bc_hi, (T)it.V[0], (T)it.V[1], (T)it.V[2], tid);
  else if (OP == OP_COMMUP)
    el_commup<T>(it.L, it.F, tid);
  else if (OP == OP_COMMMEAN)
    el_commmean<T>(it.L, it.F, it.band, tid);
  else if (OP == OP_DT_LEVEL)
    el_dt_level<T>(it.L, it.b, it.level, it.gg, it.gga, it.flags & FL_HYDRO, it.ds, it.rho0d, it.e0d,
                   it.V[0], it.V[1], it.V[2], it.bg, tid);
  else if (OP == OP_DT_FINAL)
    el_dt_finalize(it.ds, it.level, *it.fin, it.dt_fixed);
  else if (OP == OP_FORCE_LEVEL)
    el_force_level<T>(it.L, it.b, it.L.fw, it.partials, tid);
  else if (OP == OP_FORCE_FINAL)
    el_force_finalize(it.partials, it.npart, it.ds, it.ring, it.ring_cap, it.ring_pos);
  else if (OP == OP_TIME)
    el_time_advance(it.ds);
}

// Persistent work-list kernel: block b takes the contiguous chunks
// [b*nchunks/grid, (b+1)*nchunks/grid) of the concatenated items, stages the item of
// each chunk in shared memory (re-staging only when the item changes) and runs the
// op on the chunk's elements.  starts[i] is the first chunk of item i.
// (two-cell ops: at least 4 blocks per SM, so as many cells stay in flight as with
// one cell per thread at full occupancy)
template <class T, int OP, int D>
__global__ void __launch_bounds__(kBlock, cells_per_thread(OP, (int)sizeof(T)) == 2 ? 4 : 1)
    k_batch(const Item<T>* __restrict__ items,
                                                  const unsigned* __restrict__ starts, int nitems,
                                                  unsigned nchunks) {
  __shared__ __align__(16) unsigned char s_raw[sizeof(Item<T>)];
  const Item<T>& it = *reinterpret_cast<const Item<T>*>(s_raw);
  pdl_enter();
  unsigned c0 = (unsigned)((unsigned long long)nchunks * blockIdx.x / gridDim.x);
  unsigned c1 = (unsigned)((unsigned long long)nchunks * (blockIdx.x + 1) / gridDim.x);
  int cur = -1;
  for (unsigned ch = c0; ch < c1; ++ch) {
    int lo = cur < 0 ? 0 : cur, hi = nitems - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (starts[mid] <= ch)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (lo != cur) {
      __syncthreads();
      const int4* src = reinterpret_cast<const int4*>(items + lo);
      int4* dst = reinterpret_cast<int4*>(s_raw);
      for (int w = threadIdx.x; w < (int)(sizeof(Item<T>) / 16); w += kBlock) dst[w] = src[w];
      __syncthreads();
      cur = lo;
    }
    // private copy where it scalarises (global stores cannot alias it, so the
    // fields the op uses stay in registers); ops that index the item's arrays with
    // run-time indices read it from shared memory instead
    constexpr bool kLocal =
        !(OP == OP_COMPRESS || OP == OP_FRONTIER_DIFF || OP == OP_BC || OP == OP_COMMUP);
    if (kLocal) {
      const Item<T> loc = it;
      run_op<T, OP, D>(loc, (ch - starts[cur]) * kBlock + threadIdx.x);
    } else {
      run_op<T, OP, D>(it, (ch - starts[cur]) * kBlock + threadIdx.x);
    }
    __syncthreads();
  }
  pdl_exit();
}

// One work item: passed by value (kernel-parameter space), one block per chunk.
template <class T, int OP, int D>
__global__ void __launch_bounds__(kBlock) k_single(const Item<T> it) {
  pdl_enter();
  run_op<T, OP, D>(it, blockIdx.x * kBlock + threadIdx.x);
  pdl_exit();
}

// Fused sweep: one block per (column, chunk) unit; the work-list form stages the
// item as k_batch does.
template <class T, int D>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_single(const Item<T> it) {
  __shared__ __align__(16) Arith<T> s_x[2 * 3 * kSweepThreads];
  pdl_enter();
  if (skipped(it)) return;
  el_sweep<T, D>(it, blockIdx.x, s_x);
  pdl_exit();
}

template <class T, int D>
__global__ void __launch_bounds__(kSweepThreads, sizeof(T) == 4 ? 2 : 1) k_sweep_batch(const Item<T>* __restrict__ items,
                                                              const unsigned* __restrict__ starts,
                                                              int nitems, unsigned nchunks) {
  __shared__ __align__(16) Arith<T> s_x[2 * 3 * kSweepThreads];
  __shared__ __align__(16) unsigned char s_raw[sizeof(Item<T>)];
  const Item<T>& it = *reinterpret_cast<const Item<T>*>(s_raw);
  pdl_enter();
  unsigned c0 = (unsigned)((unsigned long long)nchunks * blockIdx.x / gridDim.x);
  unsigned c1 = (unsigned)((unsigned long long)nchunks * (blockIdx.x + 1) / gridDim.x);
  int cur = -1;
  for (unsigned ch = c0; ch < c1; ++ch) {
    int lo = cur < 0 ? 0 : cur, hi = nitems - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (starts[mid] <= ch)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (lo != cur) {
      __syncthreads();
      const int4* src = reinterpret_cast<const int4*>(items + lo);
      int4* dst = reinterpret_cast<int4*>(s_raw);
      for (int w = threadIdx.x; w < (int)(sizeof(Item<T>) / 16); w += kSweepThreads)
        dst[w] = src[w];
      __syncthreads();
      cur = lo;
    }
    if (!skipped(it)) el_sweep<T, D>(it, ch - starts[cur], s_x);
    __syncthreads();
  }
  pdl_exit();
}

// launch with the programmatic-stream-serialisation attribute (see pdl_enter); an
// error is left in the runtime's last-error state like that of a <<<>>> launch
template <class... P, class... A>
static void launch_pdl(void (*kernel)(P...), unsigned grid, unsigned block, cudaStream_t st,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

template <class T, int D>
static void launch_sweep(const Item<T>* items, const unsigned* starts, int nitems,
                         unsigned nchunks, unsigned grid, cudaStream_t st,
                         const Item<T>* host_item) {
  if (nitems == 1 && host_item)
    launch_pdl(k_sweep_single<T, D>, nchunks, kSweepThreads, st, *host_item);
  else
    launch_pdl(k_sweep_batch<T, D>, grid, kSweepThreads, st, items, starts, nitems, nchunks);
}

template <class T, int OP, int D>
static void launch_one(const Item<T>* items, const unsigned* starts, int nitems, unsigned nchunks,
                       unsigned grid, cudaStream_t st, const Item<T>* host_item) {
  if (nitems == 1 && host_item)
    launch_pdl(k_single<T, OP, D>, nchunks, kBlock, st, *host_item);
  else
    launch_pdl(k_batch<T, OP, D>, grid, kBlock, st, items, starts, nitems, nchunks);
}

template <class T>
int launch_batch(int op, int d, const Item<T>* items, const unsigned* starts, int nitems,
                 unsigned nchunks, unsigned grid, cudaStream_t st, const Item<T>* host_item) {
  if (nchunks == 0 || nitems == 0) return 0;
  if (grid > nchunks) grid = nchunks;
#define DFN_OP(O)                                                          \
  case O:                                                                  \
    launch_one<T, O, 0>(items, starts, nitems, nchunks, grid, st, host_item); \
    break;
#define DFN_OPD(O)                                                         \
  case O:                                                                  \
    if (d == 0) launch_one<T, O, 0>(items, starts, nitems, nchunks, grid, st, host_item); \
    if (d == 1) launch_one<T, O, 1>(items, starts, nitems, nchunks, grid, st, host_item); \
    if (d == 2) launch_one<T, O, 2>(items, starts, nitems, nchunks, grid, st, host_item); \
    break;
  switch (op) {
    DFN_OP(OP_SOURCE)
    DFN_OP(OP_COMPRESS)
    DFN_OP(OP_FRONTIER_DIFF)
    case OP_DIFFUSE:  // d = 1: with the x sweep's preparation
      if (d == 0) launch_one<T, OP_DIFFUSE, 0>(items, starts, nitems, nchunks, grid, st, host_item);
      if (d == 1) launch_one<T, OP_DIFFUSE, 1>(items, starts, nitems, nchunks, grid, st, host_item);
      break;
    DFN_OP(OP_TPREP)
    DFN_OPD(OP_TFLUX)
    DFN_OPD(OP_TMOM)
    DFN_OPD(OP_TUPDATE)
    case OP_VREC:  // d = 1: with the next sub-cycle's first kick
      if (d == 0) launch_one<T, OP_VREC, 0>(items, starts, nitems, nchunks, grid, st, host_item);
      if (d == 1) launch_one<T, OP_VREC, 1>(items, starts, nitems, nchunks, grid, st, host_item);
      break;
    DFN_OPD(OP_BC)
    DFN_OP(OP_COMMUP)
    DFN_OP(OP_COMMMEAN)
    DFN_OP(OP_DT_LEVEL)
    DFN_OP(OP_DT_FINAL)
    DFN_OP(OP_FORCE_LEVEL)
    DFN_OP(OP_FORCE_FINAL)
    DFN_OP(OP_TIME)
    DFN_OP(OP_VISC_Q)
    DFN_OP(OP_VISC_V)
    case OP_SWEEP:
      if (d == 0) launch_sweep<T, 0>(items, starts, nitems, nchunks, grid, st, host_item);
      if (d == 1) launch_sweep<T, 1>(items, starts, nitems, nchunks, grid, st, host_item);
      if (d == 2) launch_sweep<T, 2>(items, starts, nitems, nchunks, grid, st, host_item);
      break;
    default:
      return 0;
  }
#undef DFN_OP
#undef DFN_OPD
  return 1;
}

// blocks of a context's sweep kernel to aim for: those resident on the whole device
// at once (SMs x the blocks one SM holds), per state size and direction; looked up
// once
int sweep_slots(int esz, int d) {
  static int cache[2][3] = {};
  const int t = esz == 8 ? 1 : 0;
  if (cache[t][d] == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* k = nullptr;
    if (esz == 8)
      k = d == 0 ? (const void*)k_sweep_single<double, 0>
                 : d == 1 ? (const void*)k_sweep_single<double, 1>
                          : (const void*)k_sweep_single<double, 2>;
    else
      k = d == 0 ? (const void*)k_sweep_single<float, 0>
                 : d == 1 ? (const void*)k_sweep_single<float, 1>
                          : (const void*)k_sweep_single<float, 2>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kSweepThreads, 0) != cudaSuccess)
      per = 1;
    // with a single resident block per SM, several waves hide latency better than
    // long chunks (measured on the FP64 state's sweeps): keep about 600 blocks
    cache[t][d] = per >= 2 ? sms * per : 600;
  }
  return cache[t][d];
}

// elements per chunk of each op (one chunk = one block pass)
int op_chunk_elems(int op, int esz) {
  if (op == OP_DT_LEVEL) return kBlock * kDtCells;
  return op == OP_FORCE_LEVEL ? kBlock * kForceCells : kBlock * cells_per_thread(op, esz);
}

// index-space size of one item of an op (host side, from the item's views)
unsigned op_count(int op, int d, const LevelView& L, const LevelView& F, const Box& b) {
  long long n = 0;
  switch (op) {
    case OP_SOURCE: case OP_COMPRESS: case OP_DIFFUSE: case OP_TPREP: case OP_TFLUX:
    case OP_TMOM: case OP_TUPDATE: case OP_VREC: case OP_VISC_Q: case OP_VISC_V:  // is_box_op
      if (b.tile == 0) {
        n = b.count();
      } else {
        long long nt = 1;
        for (int a = 0; a < 3; ++a) {
          int e = tile_extent(b.tile, a);
          nt *= (b.hi[a] - b.lo[a] + e - 1) / e;
        }
        n = nt * 256;
      }
      break;
    case OP_SWEEP:
      n = (long long)sweep_units(b, d) * kBlock;  // one chunk per (column, chunk) unit
      break;
    case OP_FRONTIER_DIFF: n = 24LL * L.acc_slots; break;
    case OP_BC: {
      int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      n = (long long)L.s[t1] * L.s[t2] * 2 * L.G * 5;
      break;
    }
    case OP_COMMUP:  // one chunk per tile of the ghost hosts' shell
      n = cu_chunks(F.n, F.G) * kBlock;
      break;
    case OP_COMMMEAN: n = (long long)(F.n[0] >> 1) * (F.n[1] >> 1) * (F.n[2] >> 1); break;
    case OP_DT_LEVEL: case OP_FORCE_LEVEL: n = (long long)L.n[0] * L.n[1] * L.n[2]; break;
    default: n = 1; break;
  }
  // the compression kernel also sums the child's CommFlux record (fr_sums): enough
  // threads for it whatever the box (elements beyond the box decode to nothing)
  if (op == OP_COMPRESS && L.has_child && n < 18LL * L.cacc_slots) n = 18LL * L.cacc_slots;
  return (unsigned)n;
}

int force_partials_per_level(const LevelView& L) {
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  return (int)((na + kBlock * kForceCells - 1) / (kBlock * kForceCells));
}

int launch_force_weights(const LevelView& L, const Phys& P, cudaStream_t st) {
  k_force_weights<<<grid_for((long long)L.n[0] * L.n[1] * L.n[2]), kBlock, 0, st>>>(
      L, P.GM, P.eps, P.mult, L.fw);
  return 1;
}

template <class T>
int launch_init_uniform(const LevelView& L, const Phys& P, cudaStream_t st) {
  k_init_uniform<T><<<grid_for(L.nc), kBlock, 0, st>>>(L, (T)P.rho0, (T)P.e0, (T)P.V[0],
                                                        (T)P.V[1], (T)P.V[2]);
  return 1;
}

template <class T>
int launch_static_fields(const LevelView& L, const Phys& P, double lum_sigma, double* wsum,
                         double* partials, cudaStream_t st) {
  int v[3], ok = 1;
  for (int d = 0; d < 3; ++d) {
    double o = -L.lo[d] / L.dx[d];
    v[d] = (int)floor(o + 0.5);
    // a vertex on a mirror plane has four of its eight cells in the ghost layer
    if (fabs(o - v[d]) > 1e-9 || v[d] < (L.mir >> d & 1 ? 0 : 1) || v[d] > L.n[d] - 1) ok = 0;
  }
  k_static<T><<<grid_for(L.nc), kBlock, 0, st>>>(L, P.GM, P.eps, lum_sigma, ok, v[0], v[1], v[2]);
  if (lum_sigma <= 0.0) return 1;
  long long na = (long long)L.n[0] * L.n[1] * L.n[2];
  k_lum_partials<T><<<grid_for(na), kBlock, 0, st>>>(L, partials);
  k_sum_partials<<<1, kBlock, 0, st>>>(partials, (int)grid_for(na), wsum);
  return 3;
}

template <class T>
int launch_normalise_lum(const LevelView& L, const double* wsum, double mult, cudaStream_t st) {
  k_normalise_lum<T><<<grid_for(L.nc), kBlock, 0, st>>>(L, wsum, mult);
  return 1;
}

template <class T>
int launch_pack_active(const LevelView& L, int field, double* out, int full, double bgv,
                       cudaStream_t st) {
  long long n = full ? L.nc : (long long)L.n[0] * L.n[1] * L.n[2];
  k_pack<T><<<grid_for(n), kBlock, 0, st>>>(L, field, out, full, bgv);
  return 1;
}

template <class T>
int launch_unpack_active(const LevelView& L, int field, const double* in, int full, double bgv,
                         cudaStream_t st) {
  long long n = full ? L.nc : (long long)L.n[0] * L.n[1] * L.n[2];
  k_unpack<T><<<grid_for(n), kBlock, 0, st>>>(L, field, in, full, bgv);
  return 1;
}

#define DFN_INSTANTIATE(T)                                                                     \
  template int launch_batch<T>(int, int, const Item<T>*, const unsigned*, int, unsigned,       \
                               unsigned, cudaStream_t, const Item<T>*);                        \
  template int launch_init_uniform<T>(const LevelView&, const Phys&, cudaStream_t);            \
  template int launch_static_fields<T>(const LevelView&, const Phys&, double, double*,         \
                                       double*, cudaStream_t);                                 \
  template int launch_normalise_lum<T>(const LevelView&, const double*, double, cudaStream_t); \
  template int launch_pack_active<T>(const LevelView&, int, double*, int, double, cudaStream_t); \
  template int launch_unpack_active<T>(const LevelView&, int, const double*, int, double,      \
                                       cudaStream_t);

DFN_INSTANTIATE(double)
DFN_INSTANTIATE(float)

}  // namespace dfn
