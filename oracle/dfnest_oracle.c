/*
 * dfnest_oracle.c -- plain, slow, FP64 CPU oracle of the nested-mesh solver of
 * Velasco Romero & Masset (2018), Sec. 3 (numerical implementation) and Sec. 3.4
 * (dynamical-friction set-up).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py.  It shares no code with the CUDA path.
 * Compiled with -O2 -ffp-contract=off so no multiply-add is fused.
 *
 * The "omp parallel for" lines act only in a second build with -fopenmp, used to
 * time the oracle on all host cores.  Each marks a loop over planes whose
 * iterations write disjoint elements from values that no iteration of it writes, so
 * both builds compute the same bits.  Sums stay serial: the Delta t minima, the
 * force and the luminosity normalisation.  A child's frontier record is a sum too:
 * the flux loops that add into it run over pairs of planes (2p, 2p+1).  The fine
 * faces of one coarse slot lie in one pair (G is even), and within a pair the order
 * is that of the plain loops, so every slot is summed in the same order.
 *
 * Layout: every level holds (n+2G)^3 elements per field, x fastest.  rho and e are
 * cell-centred; v_d is stored at the lower d-face of the cell with the same index
 * (staggered mesh, Sec. 3.2.1 "centred and staggered quantities").
 *
 * Readings of the paper that this oracle fixes (every one is shared by the CUDA path):
 *  R1  Phi = -GM / sqrt(r^2 + eps^2): Eq. 16 prints the sign garbled; Sec. 2.1 gives
 *      the attractive potential -GM/|r|.
 *  R2  Diffusion raises e where e/rho is below its neighbours: e_i += dt (f_{i+1/2} -
 *      f_{i-1/2}) / V with f = chi rho_f (e/rho)_diff S / dx (Eqs. 19-22 print the
 *      opposite, anti-diffusive sign; Eq. 28 fixes the sign).  rho_f is the mean of
 *      the two cells (Eq. 3), or rho0 (Eqs. 19-21) when diff_face_rho = 1.
 *  R3  SubStep3 (compression heating, the p div v term of Eq. 3) is the time-centred
 *      update e <- e (1 - a)/(1 + a), a = dt (gamma-1) div v / 2, div v from the
 *      faces of v^p.  SubStep2 (artificial viscosity) is not used.
 *  R4  Level step order: S(dt/2) -> SubStep3(dt) -> luminosity(dt) -> diffusion(dt)
 *      -> transport x, y, z (dt, fluxes from v^p) -> S(dt/2)  (Eq. 15, Sec. 3.3).
 *  R5  Transport: directional sweeps x, y, z; van Leer harmonic limiter
 *      2 dl dr/(dl+dr) (0 if dl dr <= 0); time-centred upwind face values; e and
 *      momenta carried as (q/rho)* times the mass flux; staggered momenta use the
 *      mass flux averaged to their control-volume faces; v = Pi / rho_face after
 *      the three sweeps.  All fluxes of a sweep come from the state before it.
 *  R6  Every operator is applied wherever its stencil fits inside the padded array
 *      (ghost cells included).  Level 0 ghosts are filled from the boundary types
 *      once per level step; finer levels get their ghosts only from CommUp, once
 *      per parent step, so two sub-cycles run on one fill (Sec. 3.2.1): G must be
 *      at least twice the reach of one level step for the active cells to be exact.
 *  R7  CommUp: z, then y, then x 3-point van Leer-limited interpolation from the 27
 *      coarse elements around the host element; centred fields at fine offsets
 *      -1/4, +1/4 of a coarse cell.  A staggered field along its own axis has fine
 *      faces on a coarse face (copied) or midway between two (the mean of the two:
 *      a position equidistant from two coarse faces favours neither, so a
 *      mirror-symmetric state stays symmetric; the mean is exact for linear data and
 *      bounded by its neighbours).  Every fine element outside the active set is
 *      filled (for v_d the upper frontier face counts as a ghost).
 *  R8  CommMean: coarse cells within `band` layers of the contour of the covered
 *      box take the mean of their 8 fine cells; a staggered coarse face strictly
 *      inside the covered box takes the mean of its 4 coplanar fine faces when
 *      one of its two cells is in the band.  CommUp runs before CommMean.
 *  R9  CommFlux: the coarse frontier fluxes of mass, transported energy and
 *      diffusive energy are replaced by the sum over the 4 fine faces and the
 *      sub-cycles of the fine fluxes (already multiplied by area and dt).  The
 *      staggered momentum fluxes keep the coarse mass flux.
 * R10  Luminosity: each level step adds L dt_l to the level's active cells, split
 *      over the 8 cells around the vertex at the origin (Sec. 3.4) or, with
 *      lum_sigma > 0, with Gaussian weights normalised over the active cells.
 * R11  Time step: dt_l = min over active cells and axes of cfl dx_d/(cs + |v_d|),
 *      with |v_d| the larger of the two faces, and cfl_diff / (2 chi sum_d dx_d^-2);
 *      coarse step dt = min_l dt_l prod_{m<l} xi_m (Eq. 55), taken once per coarse
 *      step from the state at its start.
 * R12  Force (Eq. 18): F = GM sum_l sum_{active, uncovered} (rho - rho0) V_c (r_c)
 *      / (r^2 + eps^2)^{3/2}.  The rho0 part of Eq. 18 cancels on a region that is
 *      symmetric about the perturber; a cell is covered when its centre lies inside
 *      the child's active box.
 * R13  Level-0 boundary fill: periodic, outflow (copy of the nearest active
 *      element), inflow (background rho0, e0, V in every ghost element) or reflect
 *      (mirror, normal velocity odd with the wall face set to 0).  The two boundary
 *      faces of the normal velocity v_d (index G below the first active cell, G+n
 *      above the last) are treated alike, so the fill is mirror-symmetric, as the
 *      Sec. 3.4 problem is: under outflow both are left to the solver and the ghost
 *      faces beyond copy them; an injection face holds V on its boundary face on
 *      either side; a wall face is 0 on either side.
 * R15  SubStep2 (named in Sec. 3.3 after ZEUS) is the von Neumann-Richtmyer
 *      artificial viscosity of ZEUS (Stone & Norman 1992), applied after the first
 *      kick when av_c2 > 0 (off by default: the paper's flows are nearly linear).
 * R16  Mirror planes (the quadrant domain of Sec. 3.4): an axis whose lower domain
 *      face lies at coordinate 0 with a reflect boundary is a symmetry plane through
 *      the perturber, and the run stands for the domain unfolded across it.  Every
 *      level then starts on the plane (child offset 0 along that axis); a finer
 *      level's step starts with the reflect fill of its mirror sides, and CommUp
 *      first refreshes the parent's mirror ghosts from the parent's current state;
 *      a mirror face is no coarse/fine frontier and does not bound CommMean's band,
 *      and a coarse frontier face in the ghost layer across a mirror takes the fine
 *      flux sum of its image;
 *      the luminosity weights of R10 also cover the mirror images of active cells in
 *      the ghost layers (part of the unfolded domain; a vertex on the plane has four
 *      of its eight cells there), and Gaussian weights are normalised over the
 *      unfolded domain, 2^(mirror axes) times the active cells; the force (R12) is
 *      the unfolded one:
 *      its components along mirror axes vanish, the others are 2^(mirror axes)
 *      times the sum over the simulated part.
 */
#include "dfnest_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { RHO = 0, ENE = 1, VXF = 2 };

typedef struct {
  int n[3], G, s[3];
  size_t nc, st[3];
  double dx[3], lo[3], vol, area[3];
  int off[3]; /* lower corner of the active box in the parent's active indices */
  int mir[3]; /* mirror axes of the run (R16) */
  double* q[5];
  double* phi;
  double* lumw; /* w_c / V_c on active cells */
  double* acc[6][3];
  size_t nacc[6];
  /* scratch */
  double *vp[3], *pi[3], *eps, *w[3], *F, *Fo, *E, *P[3];
} olevel;

struct or_sim {
  int nl;
  olevel L[OR_MAX_LEVELS];
  or_params p;
  double t, dt_last, e0, V[3];
  int xi[OR_MAX_LEVELS];
  int mir[3];  /* mirror axes (R16) */
  double mult; /* copies of the simulated part in the unfolded domain */
};

static size_t idx(const olevel* L, int i, int j, int k) {
  return ((size_t)k * L->s[1] + j) * L->s[0] + i;
}

/* van Leer (1977) harmonic slope limiter */
static double vanleer(double dl, double dr) {
  double pr = dl * dr;
  if (pr <= 0.0) return 0.0;
  return 2.0 * pr / (dl + dr);
}

/* time-centred upwind value at the face between elements c-st (left) and c (right) */
static double upwind(const double* q, size_t c, size_t st, double u, double cour) {
  if (u > 0.0) {
    double sl = vanleer(q[c - st] - q[c - 2 * st], q[c] - q[c - st]);
    return q[c - st] + 0.5 * (1.0 - cour) * sl;
  } else {
    double sr = vanleer(q[c] - q[c - st], q[c + st] - q[c]);
    return q[c] - 0.5 * (1.0 + cour) * sr;
  }
}

static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

static void level_free(olevel* L) {
  for (int f = 0; f < 5; ++f) free(L->q[f]);
  free(L->phi);
  free(L->lumw);
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 3; ++b) free(L->acc[a][b]);
  for (int d = 0; d < 3; ++d) {
    free(L->vp[d]);
    free(L->pi[d]);
    free(L->w[d]);
    free(L->P[d]);
  }
  free(L->eps);
  free(L->F);
  free(L->Fo);
  free(L->E);
}

/* element kept by CommUp (R7): centred fields on the active cells; v_d on the faces
 * strictly between two active cells along d, so both frontier faces come from the
 * parent */
static int is_active_elem(const olevel* L, int field, int i, int j, int k) {
  int c[3] = {i, j, k};
  for (int d = 0; d < 3; ++d) {
    int lo = field == VXF + d ? L->G + 1 : L->G;
    if (c[d] < lo || c[d] >= L->G + L->n[d]) return 0;
  }
  return 1;
}

/* ---------------------------------------------------------------- set-up */

or_sim* or_create(int n_levels, const int n[3], const double lo[3], const double hi[3], int G,
                  const or_params* p) {
  return or_create_ground(n_levels, n, n, lo, hi, G, p);
}

or_sim* or_create_ground(int n_levels, const int n0[3], const int nf[3], const double lo[3],
                         const double hi[3], int G, const or_params* p) {
  if (n_levels < 1 || n_levels > OR_MAX_LEVELS || G < 2 || !p) return NULL;
  for (int d = 0; d < 3; ++d)
    if (n0[d] < 4 || n0[d] % 4 || nf[d] < 4 || nf[d] % 4 || !(hi[d] > lo[d])) return NULL;
  or_sim* S = (or_sim*)calloc(1, sizeof(or_sim));
  S->nl = n_levels;
  S->p = *p;
  double g = p->gamma;
  S->e0 = p->cs * p->cs * p->rho0 / (g * (g - 1.0)); /* Sec. 3.4 */
  for (int d = 0; d < 3; ++d) S->V[d] = p->mach * p->cs * p->flow_dir[d];
  for (int l = 0; l < n_levels; ++l) S->xi[l] = 2;
  S->mult = 1.0;
  for (int d = 0; d < 3; ++d) {
    S->mir[d] = lo[d] == 0.0 && p->bc[2 * d] == OR_BC_REFLECT;
    if (S->mir[d]) S->mult *= 2.0;
  }
  for (int l = 0; l < n_levels; ++l) {
    olevel* L = &S->L[l];
    const int* n = l == 0 ? n0 : nf;
    L->G = G;
    L->nc = 1;
    for (int d = 0; d < 3; ++d) {
      /* the level's box is the ground's scaled about the origin, its cell dx0 2^-l */
      double scale = ldexp((double)n[d] / n0[d], -l);
      L->mir[d] = S->mir[d];
      L->n[d] = n[d];
      L->s[d] = n[d] + 2 * G;
      L->lo[d] = lo[d] * scale;
      L->dx[d] = (hi[d] - lo[d]) * scale / n[d];
      L->nc *= (size_t)L->s[d];
    }
    L->st[0] = 1;
    L->st[1] = (size_t)L->s[0];
    L->st[2] = (size_t)L->s[0] * L->s[1];
    L->vol = L->dx[0] * L->dx[1] * L->dx[2];
    L->area[0] = L->dx[1] * L->dx[2];
    L->area[1] = L->dx[0] * L->dx[2];
    L->area[2] = L->dx[0] * L->dx[1];
    if (l > 0) {
      const olevel* Pp = &S->L[l - 1];
      for (int d = 0; d < 3; ++d) {
        double o = (L->lo[d] - Pp->lo[d]) / Pp->dx[d];
        int oi = (int)floor(o + 0.5);
        /* child must sit on parent faces, with its ghosts and the CommUp stencil
         * inside the parent's active region, or start on a mirror plane (R16) */
        int lo_ok = S->mir[d] ? oi == 0 : oi >= G / 2 + 1;
        if (fabs(o - oi) > 1e-9 || !lo_ok || oi + n[d] / 2 + G / 2 + 1 > Pp->n[d]) {
          for (int m = 0; m <= l; ++m) level_free(&S->L[m]);
          free(S);
          return NULL;
        }
        L->off[d] = oi;
      }
    }
    for (int f = 0; f < 5; ++f) L->q[f] = dalloc(L->nc);
    L->phi = dalloc(L->nc);
    L->lumw = dalloc(L->nc);
    for (int d = 0; d < 3; ++d) {
      L->vp[d] = dalloc(L->nc);
      L->pi[d] = dalloc(L->nc);
      L->w[d] = dalloc(L->nc);
      L->P[d] = dalloc(L->nc);
    }
    L->eps = dalloc(L->nc);
    L->F = dalloc(L->nc);
    L->Fo = dalloc(L->nc);
    L->E = dalloc(L->nc);
    for (int d = 0; d < 3; ++d) {
      int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      size_t na = (size_t)(n[t1] / 2) * (size_t)(n[t2] / 2);
      for (int side = 0; side < 2; ++side) {
        L->nacc[2 * d + side] = na;
        for (int b = 0; b < 3; ++b) L->acc[2 * d + side][b] = dalloc(na);
      }
    }
    /* uniform initial state (Sec. 3.4) and the static potential (Eq. 16, reading R1) */
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          size_t c = idx(L, i, j, k);
          L->q[RHO][c] = p->rho0;
          L->q[ENE][c] = S->e0;
          for (int d = 0; d < 3; ++d) L->q[VXF + d][c] = S->V[d];
          double x = L->lo[0] + (i - G + 0.5) * L->dx[0];
          double y = L->lo[1] + (j - G + 0.5) * L->dx[1];
          double z = L->lo[2] + (k - G + 0.5) * L->dx[2];
          L->phi[c] = -p->GM / sqrt(x * x + y * y + z * z + p->eps * p->eps);
        }
    /* luminosity weights (reading R10) on the active cells and on their mirror
     * images in the ghost layers, which belong to the unfolded domain (R16) */
    int w0[3];
    for (int d = 0; d < 3; ++d) w0[d] = S->mir[d] ? 0 : G;
    if (p->lum_sigma > 0.0) {
      double sum = 0.0;
      for (int k = w0[2]; k < G + n[2]; ++k)
        for (int j = w0[1]; j < G + n[1]; ++j)
          for (int i = w0[0]; i < G + n[0]; ++i) {
            double x = L->lo[0] + (i - G + 0.5) * L->dx[0];
            double y = L->lo[1] + (j - G + 0.5) * L->dx[1];
            double z = L->lo[2] + (k - G + 0.5) * L->dx[2];
            double wgt = exp(-(x * x + y * y + z * z) / (2.0 * p->lum_sigma * p->lum_sigma));
            L->lumw[idx(L, i, j, k)] = wgt;
            if (i >= G && j >= G && k >= G) sum += wgt;
          }
      /* the unfolded domain holds mult copies of every simulated cell (R16) */
      for (int k = w0[2]; k < G + n[2]; ++k)
        for (int j = w0[1]; j < G + n[1]; ++j)
          for (int i = w0[0]; i < G + n[0]; ++i) L->lumw[idx(L, i, j, k)] /= S->mult * sum * L->vol;
    } else {
      int v[3], ok = 1;
      for (int d = 0; d < 3; ++d) {
        double o = -L->lo[d] / L->dx[d];
        v[d] = (int)floor(o + 0.5);
        if (fabs(o - v[d]) > 1e-9 || v[d] < (S->mir[d] ? 0 : 1) || v[d] > n[d] - 1) ok = 0;
      }
      if (ok) /* a vertex on a mirror plane has four of its cells in the ghost layer */
        for (int c = 0; c < 8; ++c) {
          int i = G + v[0] - 1 + (c & 1), j = G + v[1] - 1 + ((c >> 1) & 1),
              k = G + v[2] - 1 + ((c >> 2) & 1);
          L->lumw[idx(L, i, j, k)] = 1.0 / (8.0 * L->vol);
        }
    }
  }
  return S;
}

void or_destroy(or_sim* S) {
  if (!S) return;
  for (int l = 0; l < S->nl; ++l) level_free(&S->L[l]);
  free(S);
}

double or_time(const or_sim* S) { return S->t; }
double or_last_dt(const or_sim* S) { return S->dt_last; }

/* ----------------------------------------------------- level-0 boundaries */

static void bc_axis(or_sim* S, olevel* L, int d, int side, int type) {
  int G = L->G, n = L->n[d];
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  for (int b = 0; b < L->s[t2]; ++b)
    for (int a = 0; a < L->s[t1]; ++a) {
      int c[3];
      c[t1] = a;
      c[t2] = b;
      for (int g = 1; g <= G; ++g) {
        for (int f = 0; f < 5; ++f) {
          int normal = (f == VXF + d);
          int dst = side == 0 ? G - g : G + n - 1 + g, src = -1;
          double sign = 1.0, fixed = 0.0;
          int use_fixed = 0;
          switch (type) {
            case OR_BC_PERIODIC:
              src = side == 0 ? dst + n : dst - n;
              break;
            case OR_BC_OUTFLOW:
              /* the nearest active element; for v_d that is the boundary face itself
               * (G or G+n), which the solver owns on both sides (R13) */
              if (normal && side == 1) {
                if (g == 1) continue;
                src = G + n;
              } else
                src = side == 0 ? G : G + n - 1;
              break;
            case OR_BC_INFLOW:
              use_fixed = 1;
              fixed = f == RHO ? S->p.rho0 : f == ENE ? S->e0 : S->V[f - VXF];
              break;
            case OR_BC_REFLECT:
              if (!normal) {
                src = side == 0 ? G - 1 + g : G + n - g;
              } else {
                sign = -1.0;
                if (side == 0)
                  src = G + g; /* face G-g mirrors face G+g about the wall face G */
                else {
                  /* faces G+n+g' mirror G+n-g'; the wall face G+n is zero */
                  int gp = dst - (G + n);
                  if (gp == 0) {
                    use_fixed = 1;
                    fixed = 0.0;
                  } else
                    src = G + n - gp;
                }
              }
              break;
          }
          c[d] = dst;
          size_t cd = idx(L, c[0], c[1], c[2]);
          if (use_fixed) {
            L->q[f][cd] = fixed;
          } else {
            c[d] = src;
            size_t cs = idx(L, c[0], c[1], c[2]);
            L->q[f][cd] = sign * L->q[f][cs];
          }
        }
      }
      /* the lower boundary face G of v_d: zero at a wall, V on an injection face (the
       * upper boundary face G+n is the g = 1 ghost element of the upper side) */
      if ((type == OR_BC_REFLECT || type == OR_BC_INFLOW) && side == 0) {
        c[d] = G;
        L->q[VXF + d][idx(L, c[0], c[1], c[2])] = type == OR_BC_INFLOW ? S->V[d] : 0.0;
      }
    }
}

void or_fill_bc(or_sim* S) {
  olevel* L = &S->L[0];
  for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side) bc_axis(S, L, d, side, S->p.bc[2 * d + side]);
}

/* ---------------------------------------------------------- source step S */

/* S(h): v_d at every face with both cells in the array gets
 * -h [ (p_i - p_{i-1}) / (dx rho_face) + (Phi_i - Phi_{i-1}) / dx ]  (Eq. 2, Eq. 15) */
static void source_step(or_sim* S, olevel* L, double h) {
  double gm1 = S->p.gamma - 1.0;
  for (int d = 0; d < 3; ++d) {
    size_t st = L->st[d];
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          if (c3[d] < 1) continue;
          size_t c = idx(L, i, j, k), m = c - st;
          double pl = gm1 * L->q[ENE][m], pr = gm1 * L->q[ENE][c];
          double rf = 0.5 * (L->q[RHO][m] + L->q[RHO][c]);
          double acc = (pr - pl) / (L->dx[d] * rf) + (L->phi[c] - L->phi[m]) / L->dx[d];
          L->q[VXF + d][c] = L->q[VXF + d][c] - h * acc;
        }
  }
}

/* SubStep2, reading R15: the von Neumann-Richtmyer artificial viscosity in the form
   of ZEUS (Stone & Norman 1992, ApJS 80, 753), whose stage names Sec. 3.3 uses.  Along
   each axis d a compressed cell (dv = v_d at its upper face - v_d at its lower face
   < 0) carries the viscous pressure q = C2 rho dv^2; every q is formed from the
   state after the first kick, then the internal energy of each cell loses
   dt q dv / dx_d (heating, since dv < 0) and the face velocity v_d gains
   -dt (q_c - q_m) / (dx_d rho_face).  The topmost cell of an axis has no upper face
   and no q; faces of index 0 are not updated (as in the kick). */
static void viscosity_step(or_sim* S, olevel* L, double dt) {
  double c2 = S->p.av_c2;
  double* q[3];
  for (int d = 0; d < 3; ++d) q[d] = (double*)calloc(L->nc, sizeof(double));
  for (int d = 0; d < 3; ++d) {
    size_t st = L->st[d];
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          if (c3[d] >= L->s[d] - 1) continue;
          size_t c = idx(L, i, j, k);
          double dv = L->q[VXF + d][c + st] - L->q[VXF + d][c];
          q[d][c] = dv < 0.0 ? c2 * L->q[RHO][c] * dv * dv : 0.0;
        }
  }
  /* heating, from the velocities before this stage */
#pragma omp parallel for
  for (int k = 0; k < L->s[2]; ++k)
    for (int j = 0; j < L->s[1]; ++j)
      for (int i = 0; i < L->s[0]; ++i) {
        int c3[3] = {i, j, k};
        size_t c = idx(L, i, j, k);
        double h = 0.0;
        for (int d = 0; d < 3; ++d) {
          if (c3[d] >= L->s[d] - 1) continue;
          double dv = L->q[VXF + d][c + L->st[d]] - L->q[VXF + d][c];
          h += q[d][c] * dv / L->dx[d];
        }
        L->q[ENE][c] = L->q[ENE][c] - dt * h;
      }
  for (int d = 0; d < 3; ++d) {
    size_t st = L->st[d];
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          if (c3[d] < 1) continue;
          size_t c = idx(L, i, j, k), m = c - st;
          double rf = 0.5 * (L->q[RHO][m] + L->q[RHO][c]);
          L->q[VXF + d][c] = L->q[VXF + d][c] - dt * (q[d][c] - q[d][m]) / (L->dx[d] * rf);
        }
  }
  for (int d = 0; d < 3; ++d) free(q[d]);
}

/* SubStep3, reading R3 */
static void compress_step(or_sim* S, olevel* L, double dt) {
  double gm1 = S->p.gamma - 1.0;
#pragma omp parallel for
  for (int k = 0; k < L->s[2] - 1; ++k)
    for (int j = 0; j < L->s[1] - 1; ++j)
      for (int i = 0; i < L->s[0] - 1; ++i) {
        size_t c = idx(L, i, j, k);
        double div = (L->q[VXF][c + L->st[0]] - L->q[VXF][c]) / L->dx[0] +
                     (L->q[VXF + 1][c + L->st[1]] - L->q[VXF + 1][c]) / L->dx[1] +
                     (L->q[VXF + 2][c + L->st[2]] - L->q[VXF + 2][c]) / L->dx[2];
        double a = 0.5 * dt * gm1 * div;
        L->q[ENE][c] = L->q[ENE][c] * (1.0 - a) / (1.0 + a);
      }
}

/* Luminosity deposit, reading R10 */
static void luminosity_step(or_sim* S, olevel* L, double dt) {
  int G = L->G, w0[3];
  for (int d = 0; d < 3; ++d) w0[d] = S->mir[d] ? 0 : G; /* mirror images too (R16) */
#pragma omp parallel for
  for (int k = w0[2]; k < G + L->n[2]; ++k)
    for (int j = w0[1]; j < G + L->n[1]; ++j)
      for (int i = w0[0]; i < G + L->n[0]; ++i) {
        size_t c = idx(L, i, j, k);
        L->q[ENE][c] = L->q[ENE][c] + S->p.L * dt * L->lumw[c];
      }
}

/* accumulator slot of a fine frontier face (child side) */
static size_t acc_index_fine(const olevel* C, int d, const int c3[3]) {
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  return (size_t)((c3[t2] - C->G) / 2) * (C->n[t1] / 2) + (c3[t1] - C->G) / 2;
}

/* fine frontier side of face c3 along d, or -1 */
static int fine_frontier_side(const olevel* C, int d, const int c3[3]) {
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2, G = C->G;
  if (c3[t1] < G || c3[t1] >= G + C->n[t1] || c3[t2] < G || c3[t2] >= G + C->n[t2]) return -1;
  if (c3[d] == G && !C->mir[d]) return 0; /* a mirror face is no frontier (R16) */
  if (c3[d] == G + C->n[d]) return 1;
  return -1;
}

/* coarse frontier side of face c3 along d (parent side), with the slot, or -1 */
static int coarse_frontier_side(const olevel* L, const olevel* C, int d, const int c3[3],
                                size_t* slot) {
  int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2, G = L->G;
  int a = c3[t1] - G - C->off[t1], b = c3[t2] - G - C->off[t2];
  /* a ghost face across a mirror plane takes the slot of its image (R16) */
  if (a < 0 && C->mir[t1]) a = -1 - a;
  if (b < 0 && C->mir[t2]) b = -1 - b;
  if (a < 0 || a >= C->n[t1] / 2 || b < 0 || b >= C->n[t2] / 2) return -1;
  int side = -1;
  if (c3[d] == G + C->off[d] && !C->mir[d]) side = 0;
  if (c3[d] == G + C->off[d] + C->n[d] / 2) side = 1;
  if (side >= 0) *slot = (size_t)b * (C->n[t1] / 2) + a;
  return side;
}

/* Thermal diffusion, Eqs. 19-22 with reading R2; frontier capture / overwrite (R9) */
static void diffusion_step(or_sim* S, olevel* L, double dt, olevel* child, int is_child) {
  double chi = S->p.chi;
  size_t nc = L->nc;
#pragma omp parallel for
  for (size_t c = 0; c < nc; ++c) L->eps[c] = L->q[ENE][c] / L->q[RHO][c];
  /* face energy moved in +d during dt: Qdt = -chi rho_f (eps_c - eps_m) / dx * A * dt */
  for (int d = 0; d < 3; ++d) {
    size_t st = L->st[d];
    double* Q = L->P[d];
    /* planes in pairs: see the note on the record at the top of this file */
#pragma omp parallel for
    for (int kp = 0; kp < (L->s[2] + 1) / 2; ++kp)
      for (int k = 2 * kp; k < 2 * kp + 2 && k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          size_t c = idx(L, i, j, k);
          if (c3[d] < 1) {
            Q[c] = 0.0;
            continue;
          }
          size_t m = c - st;
          double rf = S->p.diff_face_rho ? S->p.rho0 : 0.5 * (L->q[RHO][m] + L->q[RHO][c]);
          Q[c] = -chi * rf * (L->eps[c] - L->eps[m]) / L->dx[d] * L->area[d] * dt;
          if (is_child) {
            int side = fine_frontier_side(L, d, c3);
            if (side >= 0) L->acc[2 * d + side][2][acc_index_fine(L, d, c3)] += Q[c];
          }
          if (child) {
            size_t slot;
            int side = coarse_frontier_side(L, child, d, c3, &slot);
            if (side >= 0) Q[c] = child->acc[2 * d + side][2][slot];
          }
        }
  }
#pragma omp parallel for
  for (int k = 1; k < L->s[2] - 1; ++k)
    for (int j = 1; j < L->s[1] - 1; ++j)
      for (int i = 1; i < L->s[0] - 1; ++i) {
        size_t c = idx(L, i, j, k);
        double div = 0.0;
        for (int d = 0; d < 3; ++d) div += L->P[d][c + L->st[d]] - L->P[d][c];
        L->q[ENE][c] = L->q[ENE][c] - div / L->vol;
      }
}

/* One directional transport sweep along d (reading R5, R9). */
static void transport_sweep(or_sim* S, olevel* L, int d, double dt, olevel* child, int is_child) {
  size_t st = L->st[d], nc = L->nc;
  double* rho = L->q[RHO];
  double* e = L->q[ENE];
  double ad = L->area[d], dxd = L->dx[d];
  int sd = L->s[d];
  (void)S;
#pragma omp parallel for
  for (size_t c = 0; c < nc; ++c) L->eps[c] = e[c] / rho[c];
  for (int m = 0; m < 3; ++m)
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          size_t c = idx(L, i, j, k);
          L->w[m][c] = c3[m] >= 1 ? L->pi[m][c] / (0.5 * (rho[c - L->st[m]] + rho[c])) : 0.0;
        }
  /* mass and energy fluxes at d-faces 2 <= i_d < s_d - 1 */
  double* Fm = L->F;   /* solver's own mass flux (the momenta use this one) */
  double* Fo = L->Fo;  /* mass flux after the frontier overwrite (rho update) */
  double* Ex = L->E;   /* energy flux after the frontier overwrite (e update) */
  /* planes in pairs: see the note on the record at the top of this file */
#pragma omp parallel for
  for (int kp = 0; kp < (L->s[2] + 1) / 2; ++kp)
    for (int k = 2 * kp; k < 2 * kp + 2 && k < L->s[2]; ++k)
    for (int j = 0; j < L->s[1]; ++j)
      for (int i = 0; i < L->s[0]; ++i) {
        int c3[3] = {i, j, k};
        size_t c = idx(L, i, j, k);
        if (c3[d] < 2 || c3[d] >= sd - 1) {
          Fm[c] = 0.0;
          Fo[c] = 0.0;
          Ex[c] = 0.0;
          continue;
        }
        double u = L->vp[d][c];
        double cour = u * dt / dxd;
        double rs = upwind(rho, c, st, u, cour);
        double F = rs * u * ad * dt;
        double es = upwind(L->eps, c, st, u, cour);
        double Ee = es * F;
        Fm[c] = F;
        Fo[c] = F;
        Ex[c] = Ee;
        if (is_child) {
          int side = fine_frontier_side(L, d, c3);
          if (side >= 0) {
            size_t a = acc_index_fine(L, d, c3);
            L->acc[2 * d + side][0][a] += F;
            L->acc[2 * d + side][1][a] += Ee;
          }
        }
        if (child) {
          size_t slot;
          int side = coarse_frontier_side(L, child, d, c3, &slot);
          if (side >= 0) {
            Fo[c] = child->acc[2 * d + side][0][slot];
            Ex[c] = child->acc[2 * d + side][1][slot];
          }
        }
      }
  /* momentum fluxes */
  for (int m = 0; m < 3; ++m) {
    double* Pm = L->P[m];
    size_t sm = L->st[m];
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          size_t c = idx(L, i, j, k);
          Pm[c] = 0.0;
          if (m == d) {
            /* flux at the cell centre between faces c and c+st */
            if (c3[d] < 2 || c3[d] >= sd - 2) continue;
            double uc = 0.5 * (L->vp[d][c] + L->vp[d][c + st]);
            double Fc = 0.5 * (Fm[c] + Fm[c + st]);
            double ws = upwind(L->w[m], c + st, st, uc, uc * dt / dxd);
            Pm[c] = ws * Fc;
          } else {
            /* flux at the edge: d-face c, m-face c */
            if (c3[d] < 2 || c3[d] >= sd - 1 || c3[m] < 1) continue;
            double ue = 0.5 * (L->vp[d][c - sm] + L->vp[d][c]);
            double Fe = 0.5 * (Fm[c - sm] + Fm[c]);
            double ws = upwind(L->w[m], c, st, ue, ue * dt / dxd);
            Pm[c] = ws * Fe;
          }
        }
  }
  /* updates */
#pragma omp parallel for
  for (int k = 0; k < L->s[2]; ++k)
    for (int j = 0; j < L->s[1]; ++j)
      for (int i = 0; i < L->s[0]; ++i) {
        int c3[3] = {i, j, k};
        size_t c = idx(L, i, j, k);
        if (c3[d] >= 2 && c3[d] < sd - 2) {
          rho[c] = rho[c] - (Fo[c + st] - Fo[c]) / L->vol;
          e[c] = e[c] - (Ex[c + st] - Ex[c]) / L->vol;
        }
        for (int m = 0; m < 3; ++m) {
          if (m == d) {
            if (c3[d] >= 3 && c3[d] < sd - 2)
              L->pi[m][c] = L->pi[m][c] - (L->P[m][c] - L->P[m][c - st]) / L->vol;
          } else {
            if (c3[d] >= 2 && c3[d] < sd - 2 && c3[m] >= 1)
              L->pi[m][c] = L->pi[m][c] - (L->P[m][c + st] - L->P[m][c]) / L->vol;
          }
        }
      }
}

static void transport_step(or_sim* S, olevel* L, double dt, olevel* child, int is_child) {
  size_t nc = L->nc;
  for (int m = 0; m < 3; ++m) memcpy(L->vp[m], L->q[VXF + m], nc * sizeof(double));
  for (int m = 0; m < 3; ++m)
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          size_t c = idx(L, i, j, k);
          L->pi[m][c] =
              c3[m] >= 1 ? 0.5 * (L->q[RHO][c - L->st[m]] + L->q[RHO][c]) * L->vp[m][c] : 0.0;
        }
  for (int d = 0; d < 3; ++d) transport_sweep(S, L, d, dt, child, is_child);
  for (int m = 0; m < 3; ++m)
#pragma omp parallel for
    for (int k = 0; k < L->s[2]; ++k)
      for (int j = 0; j < L->s[1]; ++j)
        for (int i = 0; i < L->s[0]; ++i) {
          int c3[3] = {i, j, k};
          size_t c = idx(L, i, j, k);
          if (c3[m] >= 1)
            L->q[VXF + m][c] = L->pi[m][c] / (0.5 * (L->q[RHO][c - L->st[m]] + L->q[RHO][c]));
        }
}

/* One level step (reading R4) */
static void level_step(or_sim* S, int l, double dt) {
  olevel* L = &S->L[l];
  olevel* child = l + 1 < S->nl ? &S->L[l + 1] : NULL;
  int is_child = l > 0;
  if (l == 0) or_fill_bc(S);
  for (int d = 0; d < 3 && l > 0; ++d)
    if (S->mir[d]) bc_axis(S, L, d, 0, OR_BC_REFLECT); /* R16 */
  if (S->p.hydro_on) {
    source_step(S, L, 0.5 * dt);
    if (S->p.av_c2 > 0.0) viscosity_step(S, L, dt);
    compress_step(S, L, dt);
  }
  if (S->p.L != 0.0) luminosity_step(S, L, dt);
  if (S->p.chi > 0.0) diffusion_step(S, L, dt, child, is_child);
  if (S->p.hydro_on) {
    transport_step(S, L, dt, child, is_child);
    source_step(S, L, 0.5 * dt);
  }
}

/* ---------------------------------------------------- inter-level: CommUp */

static double interp3(double qm, double q0, double qp, double delta) {
  return q0 + delta * vanleer(q0 - qm, qp - q0);
}

/* one pass of R7 along an axis: centred positions at -1/4 (even) or +1/4 (odd) of
 * the host; along a staggered field's own axis the host face (even) or the mean of
 * the host face and the next one (odd) */
static double interp_pass(double qm, double q0, double qp, int own, int odd) {
  if (own) return odd ? 0.5 * (q0 + qp) : q0;
  return interp3(qm, q0, qp, odd ? 0.25 : -0.25);
}

/* floor division by 2 for possibly negative integers */
static int fdiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

void or_commup(or_sim* S, int cl) {
  olevel* Cc = &S->L[cl];
  olevel* F = &S->L[cl + 1];
  int Gf = F->G, Gc = Cc->G;
  /* the stencil may reach across a mirror plane into the parent's ghosts (R16) */
  for (int d = 0; d < 3; ++d)
    if (S->mir[d]) bc_axis(S, Cc, d, 0, OR_BC_REFLECT);
  for (int f = 0; f < 5; ++f) {
    int sa = f >= VXF ? f - VXF : -1;
#pragma omp parallel for
    for (int k = 0; k < F->s[2]; ++k)
      for (int j = 0; j < F->s[1]; ++j)
        for (int i = 0; i < F->s[0]; ++i) {
          if (is_active_elem(F, f, i, j, k)) continue;
          int c3[3] = {i, j, k}, host[3], odd[3];
          for (int a = 0; a < 3; ++a) {
            int rel = c3[a] - Gf;
            odd[a] = rel - 2 * fdiv2(rel);
            host[a] = Gc + F->off[a] + fdiv2(rel);
          }
          /* z pass: 27 -> 9, then y: 9 -> 3, then x: 3 -> 1 (Sec. 3.2.1, Fig. 2) */
          double v9[3][3], v3[3];
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              double q[3];
              for (int dz = -1; dz <= 1; ++dz)
                q[dz + 1] = Cc->q[f][idx(Cc, host[0] + dx, host[1] + dy, host[2] + dz)];
              v9[dy + 1][dx + 1] = interp_pass(q[0], q[1], q[2], sa == 2, odd[2]);
            }
          for (int dx = -1; dx <= 1; ++dx)
            v3[dx + 1] = interp_pass(v9[0][dx + 1], v9[1][dx + 1], v9[2][dx + 1], sa == 1, odd[1]);
          F->q[f][idx(F, i, j, k)] = interp_pass(v3[0], v3[1], v3[2], sa == 0, odd[0]);
        }
  }
}

/* -------------------------------------------------- inter-level: CommMean */

static int in_band(const olevel* F, int band, const int a3[3]) {
  int dist = 1 << 30;
  for (int d = 0; d < 3; ++d) {
    int lo = a3[d] - F->off[d], hi = F->off[d] + F->n[d] / 2 - 1 - a3[d];
    if (lo < 0 || hi < 0) return 0;
    if (F->mir[d]) lo = 1 << 30; /* a mirror face bounds no band (R16) */
    if (lo < dist) dist = lo;
    if (hi < dist) dist = hi;
  }
  return dist < band;
}

void or_commmean(or_sim* S, int cl) {
  olevel* Cc = &S->L[cl];
  olevel* F = &S->L[cl + 1];
  int Gc = Cc->G, Gf = F->G, band = S->p.band;
  /* centred fields: mean of 8 fine cells */
#pragma omp parallel for
  for (int c = 0; c < F->n[2] / 2; ++c)
    for (int b = 0; b < F->n[1] / 2; ++b)
      for (int a = 0; a < F->n[0] / 2; ++a) {
        int a3[3] = {a + F->off[0], b + F->off[1], c + F->off[2]};
        if (!in_band(F, band, a3)) continue;
        size_t cc = idx(Cc, Gc + a3[0], Gc + a3[1], Gc + a3[2]);
        for (int f = 0; f < 2; ++f) {
          /* pairwise: x pairs, then y, then z (exact for equal values) */
          double sz[2];
          for (int dz = 0; dz < 2; ++dz) {
            double sy[2];
            for (int dy = 0; dy < 2; ++dy) {
              size_t c0 = idx(F, Gf + 2 * a, Gf + 2 * b + dy, Gf + 2 * c + dz);
              sy[dy] = F->q[f][c0] + F->q[f][c0 + 1];
            }
            sz[dz] = sy[0] + sy[1];
          }
          Cc->q[f][cc] = 0.125 * (sz[0] + sz[1]);
        }
      }
  /* staggered fields: mean of the 4 coplanar fine faces */
  for (int sa = 0; sa < 3; ++sa) {
    int t1 = sa == 0 ? 1 : 0, t2 = sa == 2 ? 1 : 2;
#pragma omp parallel for
    for (int c = 0; c < F->n[2] / 2; ++c)
      for (int b = 0; b < F->n[1] / 2; ++b)
        for (int a = 0; a < F->n[0] / 2; ++a) {
          int r[3] = {a, b, c};
          if (r[sa] == 0) continue; /* face strictly inside the covered box */
          int a3[3] = {a + F->off[0], b + F->off[1], c + F->off[2]};
          int m3[3] = {a3[0], a3[1], a3[2]};
          m3[sa] -= 1;
          if (!in_band(F, band, a3) && !in_band(F, band, m3)) continue;
          /* pairwise: pairs along the first transverse axis, then the second */
          double sv[2];
          for (int v = 0; v < 2; ++v) {
            double pair[2];
            for (int u = 0; u < 2; ++u) {
              int fi[3];
              fi[sa] = Gf + 2 * r[sa];
              fi[t1] = Gf + 2 * r[t1] + u;
              fi[t2] = Gf + 2 * r[t2] + v;
              pair[u] = F->q[VXF + sa][idx(F, fi[0], fi[1], fi[2])];
            }
            sv[v] = pair[0] + pair[1];
          }
          Cc->q[VXF + sa][idx(Cc, Gc + a3[0], Gc + a3[1], Gc + a3[2])] = 0.25 * (sv[0] + sv[1]);
        }
  }
}

/* ------------------------------------------------------------ time step */

static double level_dt(const or_sim* S, const olevel* L) {
  const or_params* p = &S->p;
  double best = INFINITY;
  int G = L->G;
  if (p->hydro_on) {
    double gg = p->gamma * (p->gamma - 1.0);
    for (int k = G; k < G + L->n[2]; ++k)
      for (int j = G; j < G + L->n[1]; ++j)
        for (int i = G; i < G + L->n[0]; ++i) {
          size_t c = idx(L, i, j, k);
          double cs = sqrt(gg * L->q[ENE][c] / L->q[RHO][c]);
          for (int d = 0; d < 3; ++d) {
            double v0 = fabs(L->q[VXF + d][c]), v1 = fabs(L->q[VXF + d][c + L->st[d]]);
            double vm = v0 > v1 ? v0 : v1;
            double t = p->cfl * L->dx[d] / (cs + vm);
            if (t < best) best = t;
          }
        }
  }
  if (p->chi > 0.0) {
    double sinv = 0.0;
    for (int d = 0; d < 3; ++d) sinv += 1.0 / (L->dx[d] * L->dx[d]);
    double t = p->cfl_diff / (2.0 * p->chi * sinv);
    if (t < best) best = t;
  }
  return best;
}

double or_xi_search(int n, const double* dtl, const double* cost, int* xi_out) {
  double best = -1.0;
  int nw = n - 1;
  for (long word = 0; word < (1L << nw); ++word) {
    double dt = INFINITY, C = 0.0, prod = 1.0;
    for (int l = 0; l < n; ++l) {
      if (l > 0) prod *= ((word >> (l - 1)) & 1) ? 2.0 : 1.0;
      double t = dtl[l] * prod; /* Eq. 55 */
      if (t < dt) dt = t;
      C += cost[l] * prod; /* Eq. 56 */
    }
    double ratio = dt / C;
    if (ratio > best) {
      best = ratio;
      for (int l = 0; l < nw; ++l) xi_out[l] = ((word >> l) & 1) ? 2 : 1;
    }
  }
  return best;
}

double or_compute_dt(or_sim* S, double* dt_level) {
  double dtl[OR_MAX_LEVELS];
  for (int l = 0; l < S->nl; ++l) {
    dtl[l] = level_dt(S, &S->L[l]);
    if (dt_level) dt_level[l] = dtl[l];
  }
  if (S->p.xi_mode == 1 && S->nl > 1) {
    double cost[OR_MAX_LEVELS];
    for (int l = 0; l < S->nl; ++l) cost[l] = (double)S->L[l].n[0] * S->L[l].n[1] * S->L[l].n[2];
    or_xi_search(S->nl, dtl, cost, S->xi);
  }
  double dt = INFINITY, prod = 1.0;
  for (int l = 0; l < S->nl; ++l) {
    if (l > 0) prod *= S->xi[l - 1];
    double t = dtl[l] * prod;
    if (t < dt) dt = t;
  }
  if (S->p.dt_fixed > 0.0) dt = S->p.dt_fixed;
  return dt;
}

/* ------------------------------------------------------------ recursion */

static void advance(or_sim* S, int l, double dt) {
  if (l + 1 < S->nl) {
    olevel* C = &S->L[l + 1];
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 3; ++b) memset(C->acc[a][b], 0, C->nacc[a] * sizeof(double));
    for (int s = 0; s < S->xi[l]; ++s) advance(S, l + 1, dt / S->xi[l]);
  }
  level_step(S, l, dt);
  if (l + 1 < S->nl) {
    or_commup(S, l);
    or_commmean(S, l);
  }
}

void or_step(or_sim* S, int nsteps) {
  for (int n = 0; n < nsteps; ++n) {
    double dt = or_compute_dt(S, NULL);
    advance(S, 0, dt);
    S->t += dt;
    S->dt_last = dt;
  }
}

/* ------------------------------------------------------------- threads */

int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---------------------------------------------------------------- force */

void or_force(const or_sim* S, double F[3]) {
  const or_params* p = &S->p;
  F[0] = F[1] = F[2] = 0.0;
  for (int l = 0; l < S->nl; ++l) {
    const olevel* L = &S->L[l];
    const olevel* C = l + 1 < S->nl ? &S->L[l + 1] : NULL;
    int G = L->G;
    for (int k = G; k < G + L->n[2]; ++k)
      for (int j = G; j < G + L->n[1]; ++j)
        for (int i = G; i < G + L->n[0]; ++i) {
          if (C) {
            int a3[3] = {i - G, j - G, k - G}, cov = 1;
            for (int d = 0; d < 3; ++d)
              if (a3[d] < C->off[d] || a3[d] >= C->off[d] + C->n[d] / 2) cov = 0;
            if (cov) continue;
          }
          size_t c = idx(L, i, j, k);
          double x = L->lo[0] + (i - G + 0.5) * L->dx[0];
          double y = L->lo[1] + (j - G + 0.5) * L->dx[1];
          double z = L->lo[2] + (k - G + 0.5) * L->dx[2];
          double r2 = x * x + y * y + z * z + p->eps * p->eps;
          double inv3 = 1.0 / (r2 * sqrt(r2));
          double m = (L->q[RHO][c] - p->rho0) * L->vol;
          F[0] += p->GM * m * x * inv3;
          F[1] += p->GM * m * y * inv3;
          F[2] += p->GM * m * z * inv3;
        }
  }
  /* the force of the unfolded domain (R16) */
  for (int d = 0; d < 3; ++d) F[d] = S->mir[d] ? 0.0 : S->mult * F[d];
}

/* ------------------------------------------------------------- field I/O */

int or_get_field(const or_sim* S, int l, int f, double* out) {
  if (l < 0 || l >= S->nl || f < 0 || f > 4) return -1;
  const olevel* L = &S->L[l];
  size_t o = 0;
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) out[o++] = L->q[f][idx(L, i + L->G, j + L->G, k + L->G)];
  return 0;
}

int or_set_field(or_sim* S, int l, int f, const double* in) {
  if (l < 0 || l >= S->nl || f < 0 || f > 4) return -1;
  olevel* L = &S->L[l];
  size_t o = 0;
  for (int k = 0; k < L->n[2]; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) L->q[f][idx(L, i + L->G, j + L->G, k + L->G)] = in[o++];
  return 0;
}

int or_get_full(const or_sim* S, int l, int f, double* out) {
  if (l < 0 || l >= S->nl || f < 0 || f > 4) return -1;
  memcpy(out, S->L[l].q[f], S->L[l].nc * sizeof(double));
  return 0;
}

int or_set_full(or_sim* S, int l, int f, const double* in) {
  if (l < 0 || l >= S->nl || f < 0 || f > 4) return -1;
  memcpy(S->L[l].q[f], in, S->L[l].nc * sizeof(double));
  return 0;
}
