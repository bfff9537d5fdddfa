/*
 * dfnest_oracle.h -- plain FP64 CPU oracle of the nested-mesh dynamical-friction
 * solver (Velasco Romero & Masset 2018, Sec. 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares no
 * source, header or helper with the CUDA path in paper_1812_03191_gb300/.
 *
 * Every operator follows the paper's step order (Sec. 3.3 list of sub-steps,
 * Eq. 15) with the readings fixed in oracle/dfnest_oracle.c's header comment.
 */
#ifndef DFNEST_ORACLE_H
#define DFNEST_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_LEVELS 16

/* boundary types, one per domain face (-x,+x,-y,+y,-z,+z) of level 0 */
enum { OR_BC_PERIODIC = 0, OR_BC_OUTFLOW = 1, OR_BC_INFLOW = 2, OR_BC_REFLECT = 3 };

typedef struct {
  double gamma;        /* adiabatic index, p = (gamma-1) e (Sec. 2.1) */
  double rho0;         /* background density */
  double cs;           /* adiabatic sound speed of the background */
  double mach;         /* |V| / cs */
  double flow_dir[3];  /* unit vector of the gas velocity V */
  double GM;           /* perturber mass (G=1 units), Plummer potential Eq. 16 */
  double eps;          /* Plummer softening length, also used in Eq. 18 */
  double chi;          /* thermal diffusivity, Eq. 3 / Eqs. 19-22 */
  double L;            /* luminosity, energy LΔt deposited per level step (Sec. 3.4) */
  double lum_sigma;    /* 0: eight cells around the vertex; >0: Gaussian of this sigma */
  double cfl;          /* Courant number of the advective limit */
  double cfl_diff;     /* safety factor of the explicit-diffusion limit */
  double dt_fixed;     /* >0: use this coarse step instead of the CFL reduction */
  int xi_mode;         /* 0: xi=2 on every level; 1: Eq. 55-56 search each coarse step */
  int bc[6];           /* level-0 boundary types */
  int diff_face_rho;   /* 0: face density = mean of the two cells (Eq. 3); 1: rho0 (Eqs. 19-21) */
  int hydro_on;        /* 0 freezes rho and v (pure diffusion tests) */
  int band;            /* CommMean band width in coarse cells (Sec. 3.2.2) */
  double av_c2;        /* SubStep2 artificial viscosity coefficient; 0 = off (reading R15) */
} or_params;

typedef struct or_sim or_sim;

/* Build the hierarchy: level l covers [lo*2^-l, hi*2^-l] with n[3] cells and G
 * ghost layers; fill the uniform initial state (Sec. 3.4).  NULL on bad input. */
or_sim* or_create(int n_levels, const int n[3], const double lo[3], const double hi[3],
                  int G, const or_params* p);
/* Same with a ground level of n0[3] cells over [lo, hi] and finer levels of n[3]
 * cells: the cell halves from level to level, and level l >= 1 spans [lo, hi] scaled
 * about the origin by (n/n0) 2^-l per axis.  n0 = 2n gives the hierarchy of
 * Sec. 4.1.1 whose first level covers a quarter of the ground's extent. */
or_sim* or_create_ground(int n_levels, const int n0[3], const int n[3], const double lo[3],
                         const double hi[3], int G, const or_params* p);
void or_destroy(or_sim* s);

/* Advance n coarse steps (Sec. 3.3 recursion, Eq. 55 time step). */
void or_step(or_sim* s, int n_coarse_steps);
/* Time step the next coarse step would take (Eq. 55), and per-level limits. */
double or_compute_dt(or_sim* s, double* dt_level /* nullable, n_levels */);
double or_time(const or_sim* s);
double or_last_dt(const or_sim* s);

/* Force on the perturber, Eq. 18, with rho - rho0 and the covered-cell mask. */
void or_force(const or_sim* s, double F[3]);
/* threads of the OpenMP build (n > 0 sets them); the plain build returns 1 */
int or_threads(int n);

/* Active cells (n0*n1*n2, x fastest) of one field: 0 rho, 1 e, 2 vx, 3 vy, 4 vz. */
int or_get_field(const or_sim* s, int level, int field, double* out);
int or_set_field(or_sim* s, int level, int field, const double* in);
/* Whole padded array ((n+2G)^3, x fastest). */
int or_get_full(const or_sim* s, int level, int field, double* out);
int or_set_full(or_sim* s, int level, int field, const double* in);

/* Individual inter-level operators, exposed for the invariance tests. */
void or_commup(or_sim* s, int coarse_level);
void or_commmean(or_sim* s, int coarse_level);
void or_fill_bc(or_sim* s);

/* Eq. 55-56: brute force over xi in {1,2}^(n-1); returns the best dt/C and
 * writes the word to xi_out. */
double or_xi_search(int n, const double* dt_level, const double* cost, int* xi_out);

#ifdef __cplusplus
}
#endif
#endif
