// internal.h -- device-side data structures and kernel launchers of libdfnest.
//
// One level (Sec. 3: "a full mesh consists of the active cells and the ghost or
// buffer cells") is a padded box of s = n + 2G elements per axis, x fastest,
// one structure-of-arrays allocation per field.  rho and e are cell-centred,
// v_d sits on the lower d-face of the cell with the same index.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
  void* phi;          // potential at cell centres (Eq. 16)
  void* lumw;         // luminosity weight / cell volume on active cells
  double* fw;         // static force weights GM V_c / (r^2 + eps^2)^(3/2), active cells
  double* acc;        // frontier flux sums of this level as a child: [side][quantity][slot]
  int acc_slots;      // slots per (side, quantity) block
  // child geometry (coarse frontier overwrite, covered mask), has_child = 0 if none
  int has_child;
  int coff[3], cn[3];
  const double* cacc;
  int cacc_slots;
  int is_child;
};

// Scratch shared by all levels of a context (levels are advanced one at a time).
struct Scratch {
  void* pi[3];  // staggered momenta during transport
  void* eps;    // e / rho
  void* w[3];   // Pi / rho_face
  void* F;      // mass flux of the current sweep
  void* E;      // energy flux of the current sweep
  void* P[3];   // momentum fluxes of the current sweep
};

struct Box {
  int lo[3], hi[3];
  long long count() const {
    return (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
  }
};

struct Phys {
  double gamma, rho0, e0, V[3], GM, eps, chi, L, cfl, cfl_diff, dt_fixed;
  int diff_face_rho, hydro_on, band;
  int bc[6];
};

// Device scalars of a context.
struct DevScalars {
  double dt;                  // current coarse step
  double t;                   // simulated time
  double F[3];                // force after the last coarse step
  double dt_last;             // coarse step of the last completed coarse step
  unsigned long long dtmin[48];  // per-level, per-axis max of cs + |v_d| (bit patterns)
  double dtlev[16];              // per-level limits of the last reduction
  double dtl[16];                // level step of each level: dt / prod_{m<l} xi_m
  float dtf[16];                 // the same in FP32
  int unhealthy;
  int pad;
};

// ---- launchers (kernels.cu); T = double or float, all asynchronous on `st`.
// Every launcher returns the number of kernels it launched.
// dt: device pointer to this level's step in T (DevScalars::dtl or ::dtf)
template <class T> int launch_source(const LevelView& L, const Box& b, const Scratch& S,
                                     const T* dt, int write_pi, double gm1, const Phys& P,
                                     cudaStream_t st);
template <class T> int launch_compress_lum(const LevelView& L, const Box& b, const Scratch& S,
                                           const T* dt, const Phys& P, int do_ss3, int do_lum,
                                           int do_eps, cudaStream_t st);
template <class T> int launch_diffuse(const LevelView& L, const Box& b, const Scratch& S,
                                      const T* dt, const Phys& P, cudaStream_t st);
template <class T> int launch_frontier_diff(const LevelView& L, const Scratch& S, const T* dt,
                                            const Phys& P, cudaStream_t st);
template <class T> int launch_tprep(const LevelView& L, const Box& b, const Scratch& S,
                                    const Phys& P, cudaStream_t st);
template <class T> int launch_tflux(const LevelView& L, const Box& b, const Scratch& S, int d,
                                    const T* dt, const Phys& P, cudaStream_t st);
template <class T> int launch_tfrontier(const LevelView& L, const Scratch& S, int d,
                                        cudaStream_t st);
template <class T> int launch_tmom(const LevelView& L, const Box& b, const Scratch& S, int d,
                                   const T* dt, const Phys& P, cudaStream_t st);
template <class T> int launch_tupdate(const LevelView& L, const Box& b, const Scratch& S, int d,
                                      cudaStream_t st);

// kernel kinds for the timing hook (df_kernel_time / df_kernel_name)
enum KernelKind {
  K_BC = 0, K_SOURCE, K_COMPRESS, K_DIFFUSE, K_FRONTIER_DIFF, K_TPREP, K_TFLUX, K_TFRONTIER,
  K_TMOM, K_TUPDATE, K_VREC_SOURCE, K_COMMUP, K_COMMMEAN, K_DT, K_FORCE, K_OTHER, K_NKINDS
};
template <class T> int launch_vrec_source(const LevelView& L, const Box& b, const Scratch& S,
                                          const T* dt, double gm1, const Phys& P,
                                          cudaStream_t st);
template <class T> int launch_bc_fill(const LevelView& L, const Phys& P, cudaStream_t st);
template <class T> int launch_commup(const LevelView& C, const LevelView& F, cudaStream_t st);
template <class T> int launch_commmean(const LevelView& C, const LevelView& F, int band,
                                       cudaStream_t st);
template <class T> int launch_dt_level(const LevelView& L, int level, const Phys& P,
                                       DevScalars* ds, cudaStream_t st);
int launch_dt_finalize(DevScalars* ds, int n_levels, const double* prod, double dt_fixed,
                       cudaStream_t st);
template <class T> int launch_force_level(const LevelView& L, const Phys& P, double* partials,
                                          int offset, cudaStream_t st);
int force_partials_per_level(const LevelView& L);
int launch_force_weights(const LevelView& L, const Phys& P, cudaStream_t st);
int launch_force_finalize(const double* partials, int n, DevScalars* ds, double* ring,
                          int ring_cap, long long* ring_pos, cudaStream_t st);
int launch_time_advance(DevScalars* ds, cudaStream_t st);
template <class T> int launch_init_uniform(const LevelView& L, const Phys& P, cudaStream_t st);
template <class T> int launch_static_fields(const LevelView& L, const Phys& P, double lum_sigma,
                                            double* wsum, double* partials, cudaStream_t st);
template <class T> int launch_normalise_lum(const LevelView& L, const double* wsum,
                                            cudaStream_t st);
// host I/O; bgv = background value of the field (0 moves the stored deviations)
template <class T> int launch_pack_active(const LevelView& L, int field, double* out, int full,
                                          double bgv, cudaStream_t st);
template <class T> int launch_unpack_active(const LevelView& L, int field, const double* in,
                                            int full, double bgv, cudaStream_t st);

// hot-path FP64 division versus IEEE division (device arrays; max_ulp zeroed by caller)
int launch_hdiv_check(const double* a, const double* b, int n, double* max_ulp, cudaStream_t st);

// set the calling thread's last-error message (df_last_error) and return `code`
int set_error(int code, const char* fmt, ...);

}  // namespace dfn
