// bt_internal.h -- data shared by the host side (bt_host.cpp) and the CUDA
// kernels (bt_kernels.cu) of the transport library.  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>

namespace bt {

constexpr int kMaxAng = 256;     // angle bins per location
constexpr int kMaxEps = 64;      // energy groups
constexpr int kMaxMu = 64;
constexpr int kMaxFaces = 6;

enum FaceType { F_INTERNAL = 0, F_OUTFLOW_P = 1, F_OUTFLOW_Q = 2, F_REFLECT_Q = 3 };
enum Axis { AX_R = 0, AX_TH = 1, AX_PH = 2, AX_TIME = 3 };

// Geometry and momentum tables (float64, device pointers), uploaded once.
struct Tables {
  int geom, slab, periodic_th, inner_reflect, inner_zero;
  int n_r, n_th, n_zone, n_s, n_e, n_mu, n_ph, n_ang;
  int th_open;         // 2D grid on [0, theta_max < pi]: the face at theta_max is open, its
                       // incoming bins take State::fbc
  int pole;            // Gauss-Lobatto mu grid: nodes 0 and n_mu-1 are mu = -1, +1, whose
                       // n_ph cells are one direction; remapped content is spread evenly over them
  double R;            // constant ratio of consecutive group centres
  double logR;
  double dphi, dth_col;
  const double* mu;    // [n_mu] Gauss-Legendre or Gauss-Lobatto nodes, ascending
  const double* smu;   // [n_mu] sqrt(1 - mu^2)
  const double* cph;   // [n_ph] cos Phi_k
  const double* sph;   // [n_ph] sin Phi_k
  const double* dOm;   // [n_ang]
  const double* dGam;  // [n_e]
  const double* eps;   // [n_e] group centres
  const double* p3;    // [2 n_e + 3] R^(3k) for k = -(n_e+1) .. n_e+1 (dGamma ratios)
  const double* vol;   // [n_zone]
  const double* r_e;   // [n_r + 1]
  const double* r_c;   // [n_r]
  const double* th_e;  // [n_th + 1]
  const double* th_c;  // [n_th]
  const double* area_r;  // [n_th][n_r + 1] radial faces
  const double* area_t;  // [n_th + 1][n_r] polar faces (column: [1][n_r], the periodic face;
                         // edge n_th is the open face when th_open)
  const double* area_p;  // [n_th][n_r] azimuthal (periodic) faces
  const double* G_r;     // [n_th][9]       cell triad -> radial-face triad of row b
  const double* G_t;     // [n_th + 1][4][9] stencil cell k -> polar face (column: [1][4][9])
  const double* G_p;     // [n_th][4][9]    periodic image k -> azimuthal face of row b
  const int* species_kind;
  // float32 copies for the mixed-precision kernels (same roundings as a
  // per-CTA conversion): mu [n_mu]; direction n0, n1, n2 and dOmega
  // [n_ang]; dGamma, 1/dGamma, eps [n_e]; R^(3k) [2 n_e + 3]
  const float *f_mu, *f_n0, *f_n1, *f_n2, *f_dOm, *f_dGam, *f_rdGam, *f_eps, *f_p3;
};

// Per-handle mutable device state.
struct State {
  void* f;              // [s][zone][e][ang] (double or float)
  void* f_next;
  const double* v;      // [zone][3] current background
  const double* al;     // [zone]
  const double* cf;     // [zone] conformal factor
  const double* v_old;  // previous background (time remap)
  const double* al_old;
  const double* cf_old;
  const double* ka;     // [s][zone][e]
  const double* ks;
  const double* fe;
  const double* fbc;    // [s][n_r][e] imposed on the incoming bins of the open face at theta_max
  double* mom_N;        // [s][zone]
  double* mom_E;        // [s][zone]
  double* mom_P;        // [s][zone][3]
  double* out_N;        // [s][zone] outflow of the last step
  double* out_E;
  double* acc;          // [4 * n_s] cumulative N_out, E_out (+ compensation terms)
  double* red;          // scratch for reductions
  int* flag;            // [4] error flags (non-finite result, ...)
  double* qye;          // [zone] lepton-number source term of the last step
  double phase_norm;    // 1/h^3 factor of the hydro source terms
  // learned remap: per (zone, remap kind, source angle) weights of the
  // float32 path (nullptr: the exact weights are computed in the kernels)
  const void* sur_tab;
  // local time stepping (split flux form): lev [zone] levels (nullptr: one
  // global step), lts_k the substep of the macro step, dt0 the finest step,
  // lts_L the number of levels.  zlist: the zones one flux launch handles,
  // CTA i -> zone zlist[i] (nullptr: CTA i -> zone i).
  const int* lev;
  const int* zlist;
  int n_zlist;          // zones in zlist (the flux launches' grid)
  int lts_k, lts_L;
  double dt0;
};

struct LaunchCfg {
  int threads;
  size_t smem_flux;
  size_t smem_remap;
};

// Kernel entry points (bt_kernels.cu).  All enqueue on `stream`; return a
// cudaError_t as int.
int launch_time_remap(const Tables& T, const State& S, int mixed, void* stream);
// launch shape nt: threads per CTA (128, 256, 512), or kShapeSplit | threads
// (256, 512; 384 in float32 only) for the split form, whose face pass launch_flux_collide then
// launches (the zone pass is launch_zone_collide); it needs the deposit
// buffers dep (split_dep_bytes) and rec (split_rec_bytes)
constexpr int kShapeSplit = 0x10000;
int launch_flux_collide(const Tables& T, const State& S, double dt, int mixed, int nt, void* dep, void* rec,
                        void* stream);
// the zone pass of the split form (after launch_flux_collide's face pass)
int launch_zone_collide(const Tables& T, const State& S, double dt, int mixed, void* dep, void* rec, void* stream);
size_t split_dep_bytes(const Tables& T, int mixed);
size_t split_rec_bytes(const Tables& T);
int launch_totals(const Tables& T, const State& S, int mixed, double* d_out /*[2*n_s]*/, void* stream);
int launch_accumulate_outflow(const Tables& T, const State& S, void* stream);
// d_zone_rates [zone] (optional): each zone's rate, whose maximum is d_rate
int launch_max_rate(const Tables& T, const State& S, double* d_rate /*[1]*/, void* stream,
                    double* d_zone_rates = nullptr);
int launch_jhk(const Tables& T, const State& S, int mixed, double* J, double* H, double* K, void* stream);
int launch_check_finite(const Tables& T, const State& S, int mixed, void* stream);
// learned remap: features X [n][16], exact targets Y [n][27] and validity of
// the rows idx [n][3] = (zone, kind, source angle)
// learned remap: fill st.sur_tab with the network's weights (checked against
// the exact ones; tripped rows take the exact weights) for the rows the step
// reads (split != 0: the split flux form, which reads only owned faces).
// counts [2]: rows evaluated, rows tripped (uint64, accumulated).
int launch_sur_table(const Tables& T, const State& S, const float* prm, float tol, int with_time, int split,
                     void* tab, unsigned long long* counts, int grid, void* stream);
size_t sur_table_bytes(const Tables& T);
int launch_sur_samples(const Tables& T, const State& S, const int* idx, long long n, float* X, float* Y, int* valid,
                       void* stream);
size_t flux_smem_bytes(const Tables& T, int mixed, int nt);
size_t remap_smem_bytes(const Tables& T, int mixed);
int max_optin_smem();
int prepare_kernels();
int flux_occupancy(const Tables& T, int mixed, int nt);

}  // namespace bt
