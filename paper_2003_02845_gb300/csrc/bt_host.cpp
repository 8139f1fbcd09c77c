// bt_host.cpp -- host side of the transport library: configuration checks,
// float64 geometry and momentum tables (Sec. 3.1), device workspace, and the
// C ABI declared in include/bt.h.  All arithmetic of the step runs in the
// kernels of bt_kernels.cu; this file only prepares tables and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cfloat>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "bt.h"
#include "bt_internal.h"
#include "bt_mlp.h"

namespace {

thread_local std::string g_err = "no error";

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(BT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes/weights: Newton iteration on P_n from Tricomi's
// asymptotic initial guess; nodes mirrored to be exactly antisymmetric.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 1; i <= (n + 1) / 2; ++i) {
    double t = kPi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
    double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(t);
    double dp = 0.0;
    for (int it = 0; it < 60; ++it) {
      double pm = 1.0, pc = z;
      for (int k = 2; k <= n; ++k) {
        double pn = ((2.0 * k - 1.0) * z * pc - (k - 1.0) * pm) / k;
        pm = pc;
        pc = pn;
      }
      if (n == 1) { pc = z; pm = 1.0; }
      dp = n * (pm - z * pc) / (1.0 - z * z);
      double dz = pc / dp;
      z -= dz;
      if (std::fabs(dz) <= 1e-17) break;
    }
    {
      double pm = 1.0, pc = z;
      for (int k = 2; k <= n; ++k) {
        double pn = ((2.0 * k - 1.0) * z * pc - (k - 1.0) * pm) / k;
        pm = pc;
        pc = pn;
      }
      if (n == 1) { pc = z; pm = 1.0; }
      dp = n * (pm - z * pc) / (1.0 - z * z);
    }
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    x[n - i] = z;
    x[i - 1] = -z;
    w[n - i] = wi;
    w[i - 1] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

// Gauss-Lobatto nodes/weights (n >= 2): x = -1, 1 and the roots of
// q(x) = P_{N-1}(x) - x P_N(x) (N = n - 1; q is proportional to
// (1 - x^2) P_N'(x)), by Newton's method from the Chebyshev-Lobatto points;
// weights 2 / (N (N + 1) P_N(x)^2).  Nodes mirrored to be exactly
// antisymmetric.
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  const int N = n - 1;
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  w[0] = w[N] = 2.0 / (N * (N + 1.0));
  // P_{N-1}, P_N and their derivatives at z by the three-term recurrence
  auto legendre2 = [N](double z, double& pN1, double& pN, double& dN1, double& dN) {
    double p0 = 1.0, p1 = z, d0 = 0.0, d1 = 1.0;
    for (int k = 2; k <= N; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      double d2 = d0 + (2.0 * k - 1.0) * p1;   // P_k' = P_{k-2}' + (2k-1) P_{k-1}
      p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    pN1 = p0; pN = p1; dN1 = d0; dN = d1;
  };
  for (int i = 1; i <= N / 2; ++i) {
    double z = std::cos(kPi * i / N);
    double pN1, pN, dN1, dN;
    for (int it = 0; it < 60; ++it) {
      legendre2(z, pN1, pN, dN1, dN);
      const double q = pN1 - z * pN;
      const double dq = dN1 - pN - z * dN;
      const double dz = q / dq;
      z -= dz;
      if (std::fabs(dz) <= 1e-17) break;
    }
    legendre2(z, pN1, pN, dN1, dN);
    const double wi = 2.0 / (N * (N + 1.0) * pN * pN);
    x[N - i] = z; x[i] = -z;
    w[N - i] = wi; w[i] = wi;
  }
  if (n % 2 == 1) {
    double pN1, pN, dN1, dN;
    legendre2(0.0, pN1, pN, dN1, dN);
    x[N / 2] = 0.0;
    w[N / 2] = 2.0 / (N * (N + 1.0) * pN * pN);
  }
}

// local triad (r_hat, theta_hat, phi_hat) as columns, row-major E[3*m + c]
void triad(double th, double ph, double E[9]) {
  double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
  double c0[3] = {st * cp, st * sp, ct}, c1[3] = {ct * cp, ct * sp, -st}, c2[3] = {-sp, cp, 0.0};
  for (int m = 0; m < 3; ++m) { E[3 * m] = c0[m]; E[3 * m + 1] = c1[m]; E[3 * m + 2] = c2[m]; }
}

// components in the src triad -> components in the dst triad: G = E_dst^T E_src
void rotation(double ths, double phs, double thd, double phd, double* G) {
  double Es[9], Ed[9];
  triad(ths, phs, Es);
  triad(thd, phd, Ed);
  for (int m = 0; m < 3; ++m)
    for (int n = 0; n < 3; ++n) G[3 * m + n] = Ed[m] * Es[n] + Ed[3 + m] * Es[3 + n] + Ed[6 + m] * Es[6 + n];
}

// Closed forms of the flat-faced cell geometry (Sec. 3.1).
// radial face at radius r: isosceles trapezoid of the chords 2 r sin(th) sin(dph/2)
double area_r(double r, double th0, double th1, double dph) {
  double c = std::cos(0.5 * dph), s = std::sin(0.5 * dph);
  double h = r * std::hypot(c * (std::sin(th1) - std::sin(th0)), std::cos(th1) - std::cos(th0));
  return 0.5 * (2.0 * r * std::sin(th0) * s + 2.0 * r * std::sin(th1) * s) * h;
}
// polar face on the cone th: trapezoid between the chords at r0 and r1
double area_t(double r0, double r1, double th, double dph) {
  double c = std::cos(0.5 * dph), s = std::sin(0.5 * dph);
  double h = (r1 - r0) * std::hypot(std::sin(th) * c, std::cos(th));
  return 0.5 * (2.0 * r0 * std::sin(th) * s + 2.0 * r1 * std::sin(th) * s) * h;
}
// azimuthal face: difference of two triangles from the origin
double area_p(double r0, double r1, double th0, double th1) {
  return 0.5 * std::sin(th1 - th0) * (r1 * r1 - r0 * r0);
}
// cell: frustum of the pyramid with apex at the origin over the radial face
double volume(double r0, double r1, double th0, double th1, double dph) {
  double thm = 0.5 * (th0 + th1), c = std::cos(0.5 * dph);
  double h1 = c * std::cos(th0 - thm) / std::hypot(std::sin(thm), c * std::cos(thm));
  return area_r(1.0, th0, th1, dph) * h1 / 3.0 * (r1 * r1 * r1 - r0 * r0 * r0);
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Every value of p[0..n) in [lo, hi] (a NaN fails both comparisons).  The
// backgrounds of large problems are hundreds of MB per call, so the check is
// branch-free within blocks (the compiler vectorises it) and large arrays are
// split over a few host threads.
static bool block_in(const double* p, size_t n, double lo, double hi) {
  for (size_t i = 0; i < n;) {
    const size_t e = std::min(n, i + 4096);
    int ok = 1;
    for (; i < e; ++i) ok &= (p[i] >= lo) & (p[i] <= hi);
    if (!ok) return false;
  }
  return true;
}
static bool all_in(const double* p, size_t n, double lo, double hi) {
  const size_t per = size_t(1) << 21;   // elements a thread takes at least
  const size_t nt = std::min<size_t>(8, n / per);
  if (nt < 2) return block_in(p, n, lo, hi);
  std::vector<char> ok(nt, 1);
  std::vector<std::thread> th;
  const size_t chunk = (n + nt - 1) / nt;
  for (size_t t = 0; t < nt; ++t) {
    const size_t a = t * chunk, b = std::min(n, a + chunk);
    th.emplace_back([&, t, a, b] { ok[t] = block_in(p + a, b - a, lo, hi) ? 1 : 0; });
  }
  for (auto& x : th) x.join();
  for (char c : ok)
    if (!c) return false;
  return true;
}

struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    size_t o = total;
    total += (bytes + 255) & ~size_t(255);
    return o;
  }
};

}  // namespace

struct bt_handle {
  bt_config cfg;
  int mixed;
  bt::Tables tb;
  bt::State st;
  cudaStream_t stream;
  void* ws;
  bool own_ws;
  size_t ws_bytes;
  std::vector<int32_t> kinds;
  // device buffers
  double* bg[2][3];   // two background slots: v, alpha, cf
  int cur;            // index of the current background slot
  double *ka, *kaf, *ks, *fe;
  void* f[2];
  int fcur;
  double* qye;
  double* tmp;        // small device scratch (rates, totals)
  bool has_bg, remap_pending;
  int n_bg = 0;        // backgrounds set so far (capped at 2)
  int64_t launches;
  size_t nzone, nbin_total, fbytes;
  int nt;              // block size of the flux kernel (autotuned)
  std::string tune_key;
  // profiling: (kernel id, start, stop) per launch while enabled
  bool prof;
  std::vector<int> prof_id;
  std::vector<cudaEvent_t> prof_ev;
  // split form of the flux step: deposit rows and records (lazily allocated)
  void* dep = nullptr;
  void* rec = nullptr;
  // generation of the device buffers a captured step reads beyond the
  // workspace (deposit rows, learned-remap table and network): bumped
  // whenever one of them is allocated, freed or swapped, so that a batch
  // graph captured with the old buffers is never replayed
  uint64_t gen = 0;
  // local time stepping: levels [zone], the zones ordered by the level of
  // their face pass (the finest level among their owned faces) and by their
  // own level ([2][zone], device), and the prefix counts per level
  int* lev_d = nullptr;
  int* lists_d = nullptr;
  int lts_L = 0;
  std::vector<int> cnt_face, cnt_zone;
  // learned remap (bt_set_surrogate)
  bt_surrogate* sur = nullptr;
  void* sur_tab = nullptr;                    // [zone][31][n_ang] weights
  unsigned long long* sur_counts = nullptr;   // [2] rows evaluated, tripped
  float sur_tol = 0.0f;
};

// The learned remap's network: parameters, normaliser, Adam state.
struct bt_surrogate {
  cudaStream_t stream = nullptr;
  float* prm = nullptr;    // [kNParam] fp32 master parameters
  float* grad = nullptr;   // [kNParam]
  float* m = nullptr;      // Adam moments [kNTrain]
  float* v = nullptr;
  float* loss = nullptr;   // [1] loss of the last batch
  int* flag = nullptr;     // [4] device-side error flags
  double* stats = nullptr; // [32] feature sums for the normaliser
  int n_sm = 0;
  int64_t adam_t = 0;      // Adam step count
};

namespace {

// Offsets of every device buffer inside one workspace.
struct WsPlan {
  size_t tables[32];
  size_t bg[2][3], ka, ks, fe, fbc, f[2], mom_N, mom_E, mom_P, out_N, out_E, acc, red, flag, qye, tmp;
  size_t ftab;   // float32 copies of the zone-independent tables
  size_t total;
};

int plan(const bt_config* c, WsPlan& P, size_t* tab_sizes) {
  const size_t nz = (size_t)c->n_r * c->n_theta;
  const size_t ns = c->n_species, ne = c->n_eps, nang = (size_t)c->n_mu * c->n_phi;
  const size_t nth = c->n_theta;
  const size_t fel = c->precision == BT_MIXED ? 4 : 8;
  Layout L;
  size_t sizes[] = {
      (size_t)c->n_mu, (size_t)c->n_mu, (size_t)c->n_phi, (size_t)c->n_phi, nang, ne, ne, nz,
      (size_t)c->n_r + 1, (size_t)c->n_r, nth + 1, nth,
      nth * (c->n_r + 1), (nth + 1) * c->n_r, nth * c->n_r,
      nth * 9, (nth + 1) * 4 * 9, nth * 4 * 9, 2 * ne + 3};
  const int ntab = sizeof(sizes) / sizeof(sizes[0]);
  for (int i = 0; i < ntab; ++i) {
    tab_sizes[i] = sizes[i];
    P.tables[i] = L.take(8 * sizes[i]);
  }
  P.tables[ntab] = L.take(4 * ns);  // species kinds
  P.ftab = L.take(4 * ((size_t)c->n_mu + 4 * nang + 3 * ne + 2 * ne + 3));
  for (int s = 0; s < 2; ++s) {
    P.bg[s][0] = L.take(8 * 3 * nz);
    P.bg[s][1] = L.take(8 * nz);
    P.bg[s][2] = L.take(8 * nz);
  }
  P.ka = L.take(8 * ns * nz * ne);
  P.ks = L.take(8 * ns * nz * ne);
  P.fe = L.take(8 * ns * nz * ne);
  P.fbc = L.take(8 * ns * (size_t)c->n_r * ne);
  P.f[0] = L.take(fel * ns * nz * ne * nang);
  P.f[1] = L.take(fel * ns * nz * ne * nang);
  P.mom_N = L.take(8 * ns * nz);
  P.mom_E = L.take(8 * ns * nz);
  P.mom_P = L.take(8 * 3 * ns * nz);
  P.out_N = L.take(8 * ns * nz);
  P.out_E = L.take(8 * ns * nz);
  P.acc = L.take(8 * 4 * ns);
  P.red = L.take(8 * 2 * ns * nz);
  P.flag = L.take(16);
  P.qye = L.take(8 * nz);
  P.tmp = L.take(8 * (4 * ns + 8));
  P.total = L.total;
  return ntab;
}

int validate(const bt_config* c) {
  if (!c) return fail(BT_ERR_ARG, "cfg is NULL");
  if (c->geom != BT_GEOM_SPHERICAL && c->geom != BT_GEOM_SLAB) return fail(BT_ERR_ARG, "unknown geom");
  if (c->n_r < 1 || c->n_theta < 1) return fail(BT_ERR_ARG, "n_r and n_theta must be >= 1");
  if (!c->r_edges || !c->eps_edges) return fail(BT_ERR_ARG, "r_edges/eps_edges NULL");
  for (int a = 0; a < c->n_r; ++a)
    if (!(c->r_edges[a + 1] > c->r_edges[a])) return fail(BT_ERR_ARG, "r_edges must increase");
  if (c->geom == BT_GEOM_SPHERICAL && c->r_edges[0] < 0.0) return fail(BT_ERR_ARG, "r_edges[0] < 0");
  if (c->geom == BT_GEOM_SLAB && c->n_theta != 1) return fail(BT_ERR_ARG, "slab needs n_theta == 1");
  if (c->geom == BT_GEOM_SPHERICAL) {
    if (c->theta_periodic) {
      if (c->n_theta != 1) return fail(BT_ERR_ARG, "a column needs n_theta == 1");
      if (!(c->dtheta_column > 0.0 && c->dtheta_column < 1.0)) return fail(BT_ERR_ARG, "dtheta_column out of (0, 1)");
    } else if (c->n_theta < 2) {
      return fail(BT_ERR_ARG, "2D grids need n_theta >= 2");
    }
    if (!(c->dphi_wedge > 0.0 && c->dphi_wedge < 1.0)) return fail(BT_ERR_ARG, "dphi_wedge out of (0, 1)");
  }
  if (c->n_species < 1 || !c->species_kind) return fail(BT_ERR_ARG, "species");
  if (c->n_eps < 1 || c->n_eps > bt::kMaxEps) return fail(BT_ERR_ARG, "n_eps out of range");
  if (c->n_mu < 1 || c->n_mu > bt::kMaxMu || c->n_phi < 1 || c->n_mu * c->n_phi > bt::kMaxAng)
    return fail(BT_ERR_ARG, "angular grid out of range");
  for (int i = 0; i <= c->n_eps; ++i)
    if (!(c->eps_edges[i] > 0.0) || (i > 0 && !(c->eps_edges[i] > c->eps_edges[i - 1])))
      return fail(BT_ERR_ARG, "eps_edges must be positive and increasing");
  if (c->n_eps >= 2) {
    double q0 = c->eps_edges[1] / c->eps_edges[0];
    for (int i = 1; i < c->n_eps; ++i) {
      double q = c->eps_edges[i + 1] / c->eps_edges[i];
      if (std::fabs(q / q0 - 1.0) > 1e-9) return fail(BT_ERR_ARG, "eps_edges must be log-uniform");
    }
  }
  if (c->precision != BT_FP64 && c->precision != BT_MIXED) return fail(BT_ERR_ARG, "precision");
  if (c->mu_quadrature != BT_GAUSS_LEGENDRE && c->mu_quadrature != BT_GAUSS_LOBATTO)
    return fail(BT_ERR_ARG, "mu_quadrature");
  if (c->mu_quadrature == BT_GAUSS_LOBATTO && c->n_mu < 2) return fail(BT_ERR_ARG, "Gauss-Lobatto needs n_mu >= 2");
  if (!(c->theta_max >= 0.0 && c->theta_max <= kPi)) return fail(BT_ERR_ARG, "theta_max out of [0, pi]");
  if (c->theta_max > 0.0 && c->theta_max < kPi && (c->geom != BT_GEOM_SPHERICAL || c->theta_periodic))
    return fail(BT_ERR_ARG, "theta_max < pi needs a 2D spherical grid");
  return BT_OK;
}

// Autotuner cache: one "key nt" pair per line in the file named by the
// environment variable BT_TUNE_CACHE (nothing is read or written without it).
std::mutex g_tune_mutex;

std::string tune_key(const bt_config* c) {
  std::ostringstream k;
  k << "v1|" << (c->precision == BT_MIXED ? "mixed" : "fp64") << "|g" << c->geom << "|s" << c->n_species << "|e"
    << c->n_eps << "|mu" << c->n_mu << (c->mu_quadrature == BT_GAUSS_LOBATTO ? "L" : "") << "|ph" << c->n_phi
    << "|z" << (long)c->n_r * c->n_theta;
  return k.str();
}

int tune_lookup(const std::string& key) {
  const char* path = std::getenv("BT_TUNE_CACHE");
  if (!path) return 0;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  std::ifstream in(path);
  std::string k;
  int nt = 0, found = 0;
  while (in >> k >> nt)
    if (k == key) found = nt;
  return found;
}

void tune_store(const std::string& key, int nt) {
  const char* path = std::getenv("BT_TUNE_CACHE");
  if (!path) return;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  std::map<std::string, int> all;
  {
    std::ifstream in(path);
    std::string k;
    int v;
    while (in >> k >> v) all[k] = v;
  }
  all[key] = nt;
  std::ofstream out(path, std::ios::trunc);
  for (auto& kv : all) out << kv.first << " " << kv.second << "\n";
}

}  // namespace

extern "C" {

const char* bt_last_error(void) { return g_err.c_str(); }

size_t bt_workspace_bytes(const bt_config* cfg) {
  if (validate(cfg) != BT_OK) return 0;
  WsPlan P;
  size_t ts[32];
  plan(cfg, P, ts);
  return P.total;
}

// deposit buffers of the split flux step (allocated on first use)
static int ensure_split(bt_handle* h) {
  if (h->dep && h->rec) return BT_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  ++h->gen;
  if (e == cudaSuccess && !h->dep) e = cudaMalloc(&h->dep, bt::split_dep_bytes(h->tb, h->mixed));
  if (e == cudaSuccess && !h->rec) e = cudaMalloc(&h->rec, bt::split_rec_bytes(h->tb));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->dep) cudaFree(h->dep);
    if (h->rec) cudaFree(h->rec);
    h->dep = h->rec = nullptr;
    return cuda_fail(e, "split-step deposit buffers");
  }
  return BT_OK;
}
static void release_split(bt_handle* h) {
  if (!h->dep && !h->rec) return;
  ++h->gen;
  cudaStreamSynchronize(h->stream);
  if (h->dep) cudaFree(h->dep);
  if (h->rec) cudaFree(h->rec);
  h->dep = h->rec = nullptr;
}
static bool valid_shape(int nt) {
  return nt == 128 || nt == 256 || nt == 512 || nt == (bt::kShapeSplit | 256) || nt == (bt::kShapeSplit | 384) ||
         nt == (bt::kShapeSplit | 512);
}
static bool shape_fits(const bt_handle* h, int nt) {
  // the flux kernels give each angle of a row its own thread (a CTA of fewer
  // threads than angles would leave angles out)
  const int threads = nt & ~bt::kShapeSplit;
  return threads >= h->tb.n_ang &&
         (long)bt::flux_smem_bytes(h->tb, h->mixed, nt) <= (long)bt::max_optin_smem() &&
         bt::flux_occupancy(h->tb, h->mixed, nt) > 0;
}

int bt_create(const bt_config* c, void* workspace, bt_handle** out) {
  if (!out) return fail(BT_ERR_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(c);
  if (rc != BT_OK) return rc;
  bt_handle* h = new bt_handle();
  h->cfg = *c;
  h->mixed = c->precision == BT_MIXED;
  h->stream = (cudaStream_t)c->stream;
  h->kinds.assign(c->species_kind, c->species_kind + c->n_species);
  h->cfg.species_kind = h->kinds.data();
  h->cfg.r_edges = nullptr;
  h->cfg.eps_edges = nullptr;
  WsPlan P;
  size_t ts[32];
  const int ntab = plan(c, P, ts);
  h->ws_bytes = P.total;
  if (workspace) {
    if (reinterpret_cast<uintptr_t>(workspace) % 256) { delete h; return fail(BT_ERR_ARG, "workspace must be 256-byte aligned"); }
    h->ws = workspace;
    h->own_ws = false;
  } else {
    cudaError_t e = cudaMalloc(&h->ws, P.total);
    if (e != cudaSuccess) { delete h; return cuda_fail(e, "cudaMalloc(workspace)"); }
    h->own_ws = true;
  }
  char* base = static_cast<char*>(h->ws);
  auto D = [&](size_t off) { return reinterpret_cast<double*>(base + off); };

  // ---- host tables (float64)
  const int nr = c->n_r, nth = c->n_theta, ne = c->n_eps, nmu = c->n_mu, nph = c->n_phi;
  const int nang = nmu * nph;
  const size_t nz = (size_t)nr * nth;
  const bool slab = c->geom == BT_GEOM_SLAB;
  const double dph = slab ? 0.0 : c->dphi_wedge;
  // 2D polar range [0, theta_max]; below pi the face at theta_max is open
  const bool th_open = !slab && !c->theta_periodic && c->theta_max > 0.0 && c->theta_max < kPi;
  const double th_max = th_open ? c->theta_max : kPi;
  std::vector<double> mu, wmu;
  const bool lobatto = c->mu_quadrature == BT_GAUSS_LOBATTO;
  if (lobatto) gauss_lobatto(nmu, mu, wmu);
  else gauss_legendre(nmu, mu, wmu);
  std::vector<double> smu(nmu), cph(nph), sph(nph), dOm(nang), dGam(ne), eps(ne);
  for (int j = 0; j < nmu; ++j) smu[j] = std::sqrt(1.0 - mu[j] * mu[j]);
  for (int k = 0; k < nph; ++k) {
    double P_k = (k + 0.5) * 2.0 * kPi / nph;
    cph[k] = std::cos(P_k);
    sph[k] = std::sin(P_k);
  }
  for (int j = 0; j < nmu; ++j)
    for (int k = 0; k < nph; ++k) dOm[j * nph + k] = wmu[j] * 2.0 * kPi / nph;
  for (int i = 0; i < ne; ++i) {
    double a = c->eps_edges[i], b = c->eps_edges[i + 1];
    double a3 = a * a * a, b3 = b * b * b;
    dGam[i] = (b3 - a3) / 3.0;
    eps[i] = 0.75 * (b3 * b - a3 * a) / (b3 - a3);   // number-weighted mean energy of the bin
  }
  const double R = ne >= 2 ? eps[1] / eps[0] : 2.0;
  std::vector<double> r_e(c->r_edges, c->r_edges + nr + 1), r_c(nr), th_e(nth + 1), th_c(nth);
  for (int a = 0; a < nr; ++a) r_c[a] = 0.5 * (r_e[a] + r_e[a + 1]);
  if (slab) {
    th_e[0] = 0.0; th_e[1] = 0.0;
  } else if (c->theta_periodic) {
    th_e[0] = 0.5 * kPi - 0.5 * c->dtheta_column;
    th_e[1] = 0.5 * kPi + 0.5 * c->dtheta_column;
  } else {
    for (int b = 0; b <= nth; ++b) th_e[b] = th_max * b / nth;
  }
  for (int b = 0; b < nth; ++b) th_c[b] = 0.5 * (th_e[b] + th_e[b + 1]);
  std::vector<double> vol(nz), ar(nth * (nr + 1)), at((nth + 1) * nr, 0.0), ap(nth * nr, 0.0);
  std::vector<double> Gr(9 * nth, 0.0), Gt(9 * 4 * (nth + 1), 0.0), Gp(9 * 4 * nth, 0.0);
  for (int b = 0; b < nth; ++b)
    for (int a = 0; a < nr; ++a)
      vol[b * nr + a] = slab ? (r_e[a + 1] - r_e[a]) : volume(r_e[a], r_e[a + 1], th_e[b], th_e[b + 1], dph);
  for (int b = 0; b < nth; ++b)
    for (int a = 0; a <= nr; ++a)
      ar[b * (nr + 1) + a] = slab ? 1.0 : area_r(r_e[a], th_e[b], th_e[b + 1], dph);
  if (!slab) {
    const double cph2 = std::cos(0.5 * dph);
    for (int b = 0; b < nth; ++b) {
      for (int a = 0; a < nr; ++a) ap[b * nr + a] = area_p(r_e[a], r_e[a + 1], th_e[b], th_e[b + 1]);
      // radial-face triad: colatitude of the flat face's normal
      double thr = std::atan2(std::sin(th_c[b]), std::cos(th_c[b]) * cph2);
      rotation(th_c[b], 0.0, thr, 0.0, &Gr[9 * b]);
      // periodic azimuthal face of row b: images at phi = (k-1) dphi, face at dphi/2
      for (int k = 0; k < 4; ++k) rotation(th_c[b], (k - 1) * dph, th_c[b], 0.5 * dph, &Gp[9 * (4 * b + k)]);
    }
    if (c->theta_periodic) {
      const double d = c->dtheta_column, thc = th_c[0], the = thc + 0.5 * d;
      for (int a = 0; a < nr; ++a) at[a] = area_t(r_e[a], r_e[a + 1], the, dph);
      double tht = std::atan2(std::sin(the) * cph2, std::cos(the));
      for (int k = 0; k < 4; ++k) rotation(thc + (k - 1) * d, 0.0, tht, 0.0, &Gt[9 * k]);
    } else {
      for (int e = 1; e < (th_open ? nth + 1 : nth); ++e) {
        for (int a = 0; a < nr; ++a) at[e * nr + a] = area_t(r_e[a], r_e[a + 1], th_e[e], dph);
        double tht = std::atan2(std::sin(th_e[e]) * cph2, std::cos(th_e[e]));
        for (int k = 0; k < 4; ++k) {
          int bb = e - 2 + k;
          if (bb >= 0 && bb < nth) rotation(th_c[bb], 0.0, tht, 0.0, &Gt[9 * (4 * e + k)]);
        }
      }
    }
  }
  // ratios dGamma_i / dGamma_t = R^(3 (i - t)) of the log-uniform group grid
  std::vector<double> p3(2 * ne + 3);
  for (int k = -(ne + 1); k <= ne + 1; ++k) p3[k + ne + 1] = std::pow(R, 3.0 * k);
  const std::vector<double>* tabs[] = {&mu, &smu, &cph, &sph, &dOm, &dGam, &eps, &vol, &r_e, &r_c,
                                       &th_e, &th_c, &ar, &at, &ap, &Gr, &Gt, &Gp, &p3};
  for (int i = 0; i < ntab; ++i) {
    cudaError_t e = cudaMemcpyAsync(base + P.tables[i], tabs[i]->data(), 8 * ts[i], cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { bt_destroy(h); return cuda_fail(e, "upload tables"); }
  }
  cudaMemcpyAsync(base + P.tables[ntab], h->kinds.data(), 4 * c->n_species, cudaMemcpyHostToDevice, h->stream);
  // float32 copies for the mixed kernels, rounded from the same float64
  // values the kernels would otherwise convert per CTA:
  // [mu | n0 | n1 | n2 | dOmega | dGamma | 1/dGamma | eps | R^(3k)]
  std::vector<float> ft;
  ft.reserve((size_t)nmu + 4 * nang + 5 * ne + 3);
  for (int j = 0; j < nmu; ++j) ft.push_back((float)mu[j]);
  for (int q = 0; q < nang; ++q) ft.push_back((float)mu[q / nph]);
  for (int q = 0; q < nang; ++q) ft.push_back((float)(smu[q / nph] * cph[q % nph]));
  for (int q = 0; q < nang; ++q) ft.push_back((float)(smu[q / nph] * sph[q % nph]));
  for (int q = 0; q < nang; ++q) ft.push_back((float)dOm[q]);
  for (int i = 0; i < ne; ++i) ft.push_back((float)dGam[i]);
  for (int i = 0; i < ne; ++i) ft.push_back((float)(1.0 / dGam[i]));
  for (int i = 0; i < ne; ++i) ft.push_back((float)eps[i]);
  for (int k = 0; k < 2 * ne + 3; ++k) ft.push_back((float)p3[k]);
  {
    cudaError_t e = cudaMemcpyAsync(base + P.ftab, ft.data(), 4 * ft.size(), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { bt_destroy(h); return cuda_fail(e, "upload float tables"); }
  }

  bt::Tables& T = h->tb;
  T.geom = c->geom; T.slab = slab; T.periodic_th = !slab && c->theta_periodic;
  T.th_open = th_open;
  T.inner_zero = !slab && r_e[0] == 0.0; T.inner_reflect = !slab && r_e[0] > 0.0;
  T.n_r = nr; T.n_th = nth; T.n_zone = (int)nz; T.n_s = c->n_species; T.n_e = ne;
  T.n_mu = nmu; T.n_ph = nph; T.n_ang = nang;
  T.pole = lobatto && nph > 1;   // pole nodes whose Phi cells share one direction
  T.R = R; T.logR = std::log(R); T.dphi = dph; T.dth_col = T.periodic_th ? c->dtheta_column : 0.0;
  T.mu = D(P.tables[0]); T.smu = D(P.tables[1]); T.cph = D(P.tables[2]); T.sph = D(P.tables[3]);
  T.dOm = D(P.tables[4]); T.dGam = D(P.tables[5]); T.eps = D(P.tables[6]); T.vol = D(P.tables[7]);
  T.r_e = D(P.tables[8]); T.r_c = D(P.tables[9]); T.th_e = D(P.tables[10]); T.th_c = D(P.tables[11]);
  T.area_r = D(P.tables[12]); T.area_t = D(P.tables[13]); T.area_p = D(P.tables[14]);
  T.G_r = D(P.tables[15]); T.G_t = D(P.tables[16]); T.G_p = D(P.tables[17]);
  T.p3 = D(P.tables[18]);
  T.species_kind = reinterpret_cast<const int*>(base + P.tables[ntab]);
  {
    const float* fb = reinterpret_cast<const float*>(base + P.ftab);
    T.f_mu = fb; fb += nmu;
    T.f_n0 = fb; fb += nang;
    T.f_n1 = fb; fb += nang;
    T.f_n2 = fb; fb += nang;
    T.f_dOm = fb; fb += nang;
    T.f_dGam = fb; fb += ne;
    T.f_rdGam = fb; fb += ne;
    T.f_eps = fb; fb += ne;
    T.f_p3 = fb;
  }

  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < 3; ++q) h->bg[s][q] = D(P.bg[s][q]);
  h->cur = 0;
  h->ka = D(P.ka); h->ks = D(P.ks); h->fe = D(P.fe);
  h->f[0] = base + P.f[0]; h->f[1] = base + P.f[1]; h->fcur = 0;
  h->qye = D(P.qye); h->tmp = D(P.tmp);
  bt::State& S = h->st;
  S.mom_N = D(P.mom_N); S.mom_E = D(P.mom_E); S.mom_P = D(P.mom_P);
  S.out_N = D(P.out_N); S.out_E = D(P.out_E); S.acc = D(P.acc); S.red = D(P.red);
  S.flag = reinterpret_cast<int*>(base + P.flag);
  S.ka = h->ka; S.ks = h->ks; S.fe = h->fe;
  S.fbc = D(P.fbc);
  S.qye = h->qye;
  S.phase_norm = c->phase_norm;
  h->nzone = nz;
  h->nbin_total = (size_t)c->n_species * nz * ne * nang;
  h->fbytes = h->nbin_total * (h->mixed ? 4 : 8);
  cudaMemsetAsync(h->f[0], 0, h->fbytes, h->stream);
  cudaMemsetAsync(S.acc, 0, 8 * 4 * c->n_species, h->stream);
  cudaMemsetAsync(D(P.fbc), 0, 8 * (size_t)c->n_species * nr * ne, h->stream);
  cudaMemsetAsync(S.flag, 0, 16, h->stream);
  cudaMemsetAsync(S.mom_N, 0, 8 * c->n_species * nz, h->stream);
  cudaMemsetAsync(S.mom_E, 0, 8 * c->n_species * nz, h->stream);
  cudaMemsetAsync(S.mom_P, 0, 8 * 3 * c->n_species * nz, h->stream);
  cudaMemsetAsync(h->qye, 0, 8 * nz, h->stream);
  h->launches = 0;
  h->prof = false;
  h->has_bg = false;
  h->remap_pending = false;
  // launch shape: cached autotuner choice, else 256 threads per CTA
  {
    int pe = bt::prepare_kernels();
    if (pe) { bt_destroy(h); return cuda_fail((cudaError_t)pe, "cudaFuncSetAttribute"); }
  }
  h->tune_key = tune_key(c);
  // launch shape: the autotuner's cached choice if it fits, else the first
  // of fused/256, split/256, split/512, fused/512, fused/128 that fits (the
  // split form's passes need less shared memory per CTA than the fused one)
  h->nt = 0;
  {
    const int S = bt::kShapeSplit;
    const int order[6] = {tune_lookup(h->tune_key), 256, S | 256, S | 512, 512, 128};
    for (int nt : order) {
      if (!valid_shape(nt) || !shape_fits(h, nt)) continue;
      if ((nt & S) && ensure_split(h) != BT_OK) continue;
      h->nt = nt;
      break;
    }
  }
  // shared memory per CTA must fit the opt-in limit
  int lim = bt::max_optin_smem();
  size_t need = bt::remap_smem_bytes(T, h->mixed);
  if (h->nt == 0) need = std::max(need, bt::flux_smem_bytes(T, h->mixed, 256));
  if (h->nt == 0 || (long)need > (long)lim) {
    bt_destroy(h);
    return fail(BT_ERR_ARG, "problem needs " + std::to_string(need) + " bytes of shared memory per CTA (limit " +
                                std::to_string(lim) + ")");
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) { bt_destroy(h); return cuda_fail(e, "bt_create"); }
  *out = h;
  return BT_OK;
}

static void prof_clear(bt_handle* h) {
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  h->prof_ev.clear();
  h->prof_id.clear();
}

// record an event pair around one launch while profiling is on
struct ProfScope {
  bt_handle* h;
  int id;
  cudaEvent_t a = nullptr;
  ProfScope(bt_handle* hh, int kid) : h(hh), id(kid) {
    if (!h->prof) return;
    cudaEventCreate(&a);
    cudaEventRecord(a, h->stream);
  }
  ~ProfScope() {
    if (!h->prof) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, h->stream);
    h->prof_ev.push_back(a);
    h->prof_ev.push_back(b);
    h->prof_id.push_back(id);
  }
};

int bt_destroy(bt_handle* h) {
  if (!h) return BT_OK;
  prof_clear(h);
  if (h->sur_tab) cudaFree(h->sur_tab);
  if (h->sur_counts) cudaFree(h->sur_counts);
  if (h->dep) cudaFree(h->dep);
  if (h->rec) cudaFree(h->rec);
  if (h->lev_d) cudaFree(h->lev_d);
  if (h->lists_d) cudaFree(h->lists_d);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  delete h;
  return BT_OK;
}

static int copy_in(bt_handle* h, int mem, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, mem == BT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->stream);
  return e == cudaSuccess ? BT_OK : cuda_fail(e, "copy in");
}

int bt_set_background(bt_handle* h, int mem, const double* rho, const double* T, const double* Ye,
                      const double* v, const double* alpha, const double* phi, const double* shift,
                      const double* kappa_a, const double* kappa_s, const double* f_eq) {
  (void)rho; (void)T; (void)Ye;
  if (!h || !v || !alpha || !phi || !kappa_a || !kappa_s || !f_eq) return fail(BT_ERR_ARG, "NULL background array");
  if (mem != BT_MEM_HOST && mem != BT_MEM_DEVICE) return fail(BT_ERR_ARG, "mem");
  const size_t nz = h->nzone, no = (size_t)h->cfg.n_species * nz * h->cfg.n_eps;
  if (mem == BT_MEM_HOST) {
    if (!finite_all(v, 3 * nz) || !finite_all(alpha, nz) || !finite_all(phi, nz) ||
        !all_in(f_eq, no, -DBL_MAX, DBL_MAX))
      return fail(BT_ERR_BACKGROUND, "non-finite background value");
    // opacities: finite and non-negative, in one pass
    if (!all_in(kappa_a, no, 0.0, DBL_MAX) || !all_in(kappa_s, no, 0.0, DBL_MAX)) {
      if (!finite_all(kappa_a, no) || !finite_all(kappa_s, no))
        return fail(BT_ERR_BACKGROUND, "non-finite background value");
      return fail(BT_ERR_BACKGROUND, "negative opacity");
    }
    for (size_t z = 0; z < nz; ++z) {
      if (!(alpha[z] > 0.0) || !(phi[z] > 0.0)) return fail(BT_ERR_BACKGROUND, "alpha and phi must be > 0");
      double v2 = v[3 * z] * v[3 * z] + v[3 * z + 1] * v[3 * z + 1] + v[3 * z + 2] * v[3 * z + 2];
      if (!(v2 < 1.0)) return fail(BT_ERR_BACKGROUND, "|v| must be < 1");
      if (shift && (shift[3 * z] != 0.0 || shift[3 * z + 1] != 0.0 || shift[3 * z + 2] != 0.0))
        return fail(BT_ERR_BACKGROUND, "non-zero shift is not supported");
    }
  }
  int nxt = h->has_bg ? 1 - h->cur : h->cur;
  int rc;
  if ((rc = copy_in(h, mem, h->bg[nxt][0], v, 8 * 3 * nz)) != BT_OK) return rc;
  if ((rc = copy_in(h, mem, h->bg[nxt][1], alpha, 8 * nz)) != BT_OK) return rc;
  if ((rc = copy_in(h, mem, h->bg[nxt][2], phi, 8 * nz)) != BT_OK) return rc;
  if ((rc = copy_in(h, mem, h->ka, kappa_a, 8 * no)) != BT_OK) return rc;
  if ((rc = copy_in(h, mem, h->ks, kappa_s, 8 * no)) != BT_OK) return rc;
  if ((rc = copy_in(h, mem, h->fe, f_eq, 8 * no)) != BT_OK) return rc;
  if (h->has_bg) h->remap_pending = true;
  h->cur = nxt;
  h->has_bg = true;
  if (h->n_bg < 2) ++h->n_bg;
  return BT_OK;
}

int bt_set_boundary(bt_handle* h, int mem, const double* f_boundary) {
  if (!h || !f_boundary) return fail(BT_ERR_ARG, "NULL");
  if (mem != BT_MEM_HOST && mem != BT_MEM_DEVICE) return fail(BT_ERR_ARG, "mem");
  if (!h->tb.th_open) return fail(BT_ERR_ARG, "the grid has no open face at theta_max");
  const size_t n = (size_t)h->cfg.n_species * h->cfg.n_r * h->cfg.n_eps;
  if (mem == BT_MEM_HOST && !finite_all(f_boundary, n)) return fail(BT_ERR_BACKGROUND, "non-finite boundary value");
  return copy_in(h, mem, const_cast<double*>(h->st.fbc), f_boundary, 8 * n);
}

int bt_set_f(bt_handle* h, int mem, const void* f) {
  if (!h || !f) return fail(BT_ERR_ARG, "NULL");
  int rc = copy_in(h, mem, h->f[h->fcur], f, h->fbytes);
  if (rc == BT_OK) h->remap_pending = false;
  return rc;
}

static int check_flag(bt_handle* h) {
  int flag[4];
  cudaError_t e = cudaMemcpyAsync(flag, h->st.flag, 16, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  if (flag[1]) return fail(BT_ERR_TIMEOUT, "a device-side wait for an asynchronous copy gave up");
  if (flag[0]) return fail(BT_ERR_NUMERIC, "a step produced a non-finite value");
  return BT_OK;
}

int bt_get_f(bt_handle* h, int mem, void* f) {
  if (!h || !f) return fail(BT_ERR_ARG, "NULL");
  cudaError_t e = cudaMemcpyAsync(f, h->f[h->fcur], h->fbytes,
                                  mem == BT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_get_f");
  return check_flag(h);
}

static void bind_state(bt_handle* h) {
  bt::State& S = h->st;
  int old = 1 - h->cur;
  S.v = h->bg[h->cur][0]; S.al = h->bg[h->cur][1]; S.cf = h->bg[h->cur][2];
  S.v_old = h->bg[old][0]; S.al_old = h->bg[old][1]; S.cf_old = h->bg[old][2];
  S.f = h->f[h->fcur];
  S.f_next = h->f[1 - h->fcur];
  S.sur_tab = h->sur ? h->sur_tab : nullptr;
}

int bt_max_dt(bt_handle* h, double cfl, double* dt_out) {
  if (!h || !dt_out) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_max_dt before bt_set_background");
  bind_state(h);
  int e = bt::launch_max_rate(h->tb, h->st, h->tmp, h->stream);
  h->launches += 1;
  if (e) return cuda_fail((cudaError_t)e, "max_rate");
  double rate = 0.0;
  cudaError_t ce = cudaMemcpyAsync(&rate, h->tmp, 8, cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_max_dt");
  if (!(rate > 0.0)) return fail(BT_ERR_STATE, "zero transport rate");
  *dt_out = cfl / rate;
  return BT_OK;
}

// Enqueue one step's kernels on h->stream (also used inside graph capture).
static int step_enqueue(bt_handle* h, double dt) {
  bind_state(h);
  int e;
  if (h->sur) {
    ProfScope ps(h, BT_K_SUR_TABLE);
    e = bt::launch_sur_table(h->tb, h->st, h->sur->prm, h->sur_tol, h->remap_pending ? 1 : 0,
                             (h->nt & bt::kShapeSplit) ? 1 : 0, h->sur_tab, h->sur_counts, 4 * h->sur->n_sm,
                             h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "learned remap table");
  }
  if (h->remap_pending) {
    ProfScope ps(h, BT_K_TIME_REMAP);
    e = bt::launch_time_remap(h->tb, h->st, h->mixed, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "time remap");
    h->remap_pending = false;
  }
  {
    ProfScope ps(h, BT_K_FLUX);
    e = bt::launch_flux_collide(h->tb, h->st, dt, h->mixed, h->nt, h->dep, h->rec, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "flux/collide");
  }
  if (h->nt & bt::kShapeSplit) {
    ProfScope ps(h, BT_K_ZONE);
    e = bt::launch_zone_collide(h->tb, h->st, dt, h->mixed, h->dep, h->rec, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "zone collide");
  }
  {
    ProfScope ps(h, BT_K_OUTFLOW);
    e = bt::launch_accumulate_outflow(h->tb, h->st, h->stream);
    h->launches += 2;
    if (e) return cuda_fail((cudaError_t)e, "outflow");
  }
  h->fcur = 1 - h->fcur;
  return BT_OK;
}

int bt_step(bt_handle* h, double dt) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_step before bt_set_background");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(BT_ERR_DT, "dt must be positive and finite");
  return step_enqueue(h, dt);
}

// ---------------------------------------------------------------------------
// Local time stepping (Sec. 5): zone z steps with dt0 2^lev[z]
// ---------------------------------------------------------------------------
int bt_set_levels(bt_handle* h, const int32_t* levels, int n_levels) {
  if (!h || !levels) return fail(BT_ERR_ARG, "NULL");
  if (n_levels < 1 || n_levels > 16) return fail(BT_ERR_ARG, "n_levels out of [1, 16]");
  const int nr = h->cfg.n_r, nth = h->cfg.n_theta, nz = (int)h->nzone;
  for (int z = 0; z < nz; ++z)
    if (levels[z] < 0 || levels[z] >= n_levels) return fail(BT_ERR_ARG, "level out of [0, n_levels)");
  const bool polar = h->cfg.geom == BT_GEOM_SPHERICAL && !h->cfg.theta_periodic && nth > 1;
  // the face pass of a zone runs when any face it owns is due: its outer
  // radial face and (2D) upper polar face reach the next zone; the others
  // are its own
  std::vector<int> lmin(nz);
  for (int z = 0; z < nz; ++z) {
    const int a = z % nr, b = z / nr;
    int l = levels[z];
    if (a + 1 < nr) l = std::min(l, (int)levels[z + 1]);
    if (polar && b + 1 < nth) l = std::min(l, (int)levels[z + nr]);
    lmin[z] = l;
  }
  std::vector<int> lists(2 * (size_t)nz);
  h->cnt_face.assign(n_levels, 0);
  h->cnt_zone.assign(n_levels, 0);
  for (int z = 0; z < nz; ++z) { ++h->cnt_face[lmin[z]]; ++h->cnt_zone[levels[z]]; }
  for (int l = 1; l < n_levels; ++l) { h->cnt_face[l] += h->cnt_face[l - 1]; h->cnt_zone[l] += h->cnt_zone[l - 1]; }
  {
    std::vector<int> pf(n_levels, 0), pz(n_levels, 0);
    for (int l = 1; l < n_levels; ++l) { pf[l] = h->cnt_face[l - 1]; pz[l] = h->cnt_zone[l - 1]; }
    for (int z = 0; z < nz; ++z) {   // stable: zones keep their order within a level
      lists[pf[lmin[z]]++] = z;
      lists[nz + pz[levels[z]]++] = z;
    }
  }
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && !h->lev_d) e = cudaMalloc(&h->lev_d, sizeof(int) * nz);
  if (e == cudaSuccess && !h->lists_d) e = cudaMalloc(&h->lists_d, sizeof(int) * 2 * (size_t)nz);
  if (e == cudaSuccess) e = cudaMemcpy(h->lev_d, levels, sizeof(int) * nz, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->lists_d, lists.data(), sizeof(int) * 2 * (size_t)nz, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "bt_set_levels");
  h->lts_L = n_levels;
  return BT_OK;
}

int bt_lts_levels(bt_handle* h, double cfl, int max_levels, double* dt0, int32_t* levels) {
  if (!h || !dt0) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_lts_levels before bt_set_background");
  if (max_levels < 1 || max_levels > 16) return fail(BT_ERR_ARG, "max_levels out of [1, 16]");
  const int nr = h->cfg.n_r, nth = h->cfg.n_theta, nz = (int)h->nzone;
  bind_state(h);
  double* zr = nullptr;
  cudaError_t ce = cudaMallocAsync(reinterpret_cast<void**>(&zr), sizeof(double) * nz, h->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_lts_levels");
  int e = bt::launch_max_rate(h->tb, h->st, h->tmp, h->stream, zr);
  h->launches += 1;
  std::vector<double> rate(nz);
  double mx = 0.0;
  if (!e) ce = cudaMemcpyAsync(rate.data(), zr, sizeof(double) * nz, cudaMemcpyDeviceToHost, h->stream);
  if (!e && ce == cudaSuccess) ce = cudaMemcpyAsync(&mx, h->tmp, 8, cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(zr, h->stream);
  if (!e && ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (e) return cuda_fail((cudaError_t)e, "zone rates");
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_lts_levels");
  if (!(mx > 0.0)) return fail(BT_ERR_STATE, "zero transport rate");
  // the finest step is the global Courant step; a zone takes the largest
  // dt0 2^l within its own limit cfl / rate
  std::vector<int32_t> lev(nz);
  for (int z = 0; z < nz; ++z) {
    int l = 0;
    while (l + 1 < max_levels && rate[z] * (double)(1 << (l + 1)) <= mx) ++l;
    lev[z] = l;
  }
  // neighbours (radial, and polar on 2D grids) differ by one level at most
  const bool polar = h->cfg.geom == BT_GEOM_SPHERICAL && !h->cfg.theta_periodic && nth > 1;
  for (bool changed = true; changed;) {
    changed = false;
    for (int z = 0; z < nz; ++z) {
      const int a = z % nr, b = z / nr;
      int l = lev[z];
      if (a > 0) l = std::min(l, lev[z - 1] + 1);
      if (a + 1 < nr) l = std::min(l, lev[z + 1] + 1);
      if (polar && b > 0) l = std::min(l, lev[z - nr] + 1);
      if (polar && b + 1 < nth) l = std::min(l, lev[z + nr] + 1);
      if (l != lev[z]) { lev[z] = l; changed = true; }
    }
  }
  int top = 0;
  for (int z = 0; z < nz; ++z) top = std::max(top, (int)lev[z]);
  int rc = bt_set_levels(h, lev.data(), top + 1);
  if (rc != BT_OK) return rc;
  *dt0 = cfl / mx;
  if (levels) std::copy(lev.begin(), lev.end(), levels);
  return BT_OK;
}

int bt_n_levels(const bt_handle* h) { return h ? h->lts_L : 0; }

int bt_step_lts(bt_handle* h, double dt0) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_step_lts before bt_set_background");
  if (!h->lev_d) return fail(BT_ERR_STATE, "bt_step_lts before bt_set_levels / bt_lts_levels");
  if (h->sur) return fail(BT_ERR_ARG, "the learned remap does not run with local time stepping");
  if (!(dt0 > 0.0) || !std::isfinite(dt0)) return fail(BT_ERR_DT, "dt0 must be positive and finite");
  const int S = bt::kShapeSplit;
  const int nt = (h->nt & S) ? h->nt : (S | 256);   // the split form computes each face once
  if (!shape_fits(h, nt)) return fail(BT_ERR_ARG, "the split form does not fit this problem");
  int rc = ensure_split(h);
  if (rc != BT_OK) return rc;
  bind_state(h);
  int e;
  if (h->remap_pending) {
    e = bt::launch_time_remap(h->tb, h->st, h->mixed, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "time remap");
    h->remap_pending = false;
  }
  // zones step at different times: f is updated in place (a zone pass writes
  // only its own zones, after the face pass that read them)
  bt::State st = h->st;
  st.f_next = st.f;
  const size_t nsz = (size_t)h->cfg.n_species * h->nzone;
  cudaMemsetAsync(st.mom_N, 0, 8 * nsz, h->stream);
  cudaMemsetAsync(st.mom_E, 0, 8 * nsz, h->stream);
  cudaMemsetAsync(st.mom_P, 0, 8 * 3 * nsz, h->stream);
  cudaMemsetAsync(st.out_N, 0, 8 * nsz, h->stream);
  cudaMemsetAsync(st.out_E, 0, 8 * nsz, h->stream);
  cudaMemsetAsync(h->qye, 0, 8 * h->nzone, h->stream);
  st.lev = h->lev_d;
  st.dt0 = dt0;
  st.lts_L = h->lts_L;
  const int L = h->lts_L, K = 1 << (L - 1);
  for (int k = 0; k < K; ++k) {
    st.lts_k = k;
    // a level-l face or zone starts a step at multiples of 2^l, ends one
    // before the next multiple: the due ones form a prefix of the lists
    int lf = L - 1, lz = 0;
    if (k > 0) { lf = 0; while (lf < L - 1 && (k % (1 << (lf + 1))) == 0) ++lf; }
    while (lz < L - 1 && ((k + 1) % (1 << (lz + 1))) == 0) ++lz;
    st.zlist = h->lists_d;
    st.n_zlist = h->cnt_face[lf];
    e = bt::launch_flux_collide(h->tb, st, dt0, h->mixed, nt, h->dep, h->rec, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "face pass (local time stepping)");
    st.zlist = h->lists_d + h->nzone;
    st.n_zlist = h->cnt_zone[lz];
    e = bt::launch_zone_collide(h->tb, st, dt0, h->mixed, h->dep, h->rec, h->stream);
    h->launches += 1;
    if (e) return cuda_fail((cudaError_t)e, "zone pass (local time stepping)");
  }
  st.zlist = nullptr;
  st.lev = nullptr;
  e = bt::launch_accumulate_outflow(h->tb, st, h->stream);
  h->launches += 2;
  if (e) return cuda_fail((cudaError_t)e, "outflow");
  return BT_OK;
}

int bt_autotune(bt_handle* h, double dt, int* chosen_nt) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_autotune before bt_set_background");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(BT_ERR_DT, "dt must be positive and finite");
  bind_state(h);
  const int S = bt::kShapeSplit;
  const int cand[6] = {128, 256, 512, S | 256, S | 384, S | 512};
  float best = 0.f;
  int best_nt = h->nt;
  // the trial launches write the per-zone moments and outflow of a step that
  // is never taken: keep the last step's copies and put them back afterwards
  const size_t nsz = (size_t)h->cfg.n_species * h->nzone;
  struct Keep { void* buf; size_t bytes; } keep[6] = {
      {h->st.mom_N, 8 * nsz}, {h->st.mom_E, 8 * nsz}, {h->st.mom_P, 8 * 3 * nsz},
      {h->st.out_N, 8 * nsz}, {h->st.out_E, 8 * nsz}, {h->qye, 8 * h->nzone}};
  size_t keep_bytes = 0;
  for (const Keep& k : keep) keep_bytes += k.bytes;
  char* saved = nullptr;
  {
    cudaError_t ce = cudaMallocAsync(reinterpret_cast<void**>(&saved), keep_bytes, h->stream);
    if (ce != cudaSuccess) { cudaGetLastError(); return cuda_fail(ce, "autotune: moment copies"); }
    size_t o = 0;
    for (const Keep& k : keep) {
      cudaMemcpyAsync(saved + o, k.buf, k.bytes, cudaMemcpyDeviceToDevice, h->stream);
      o += k.bytes;
    }
  }
  auto restore = [&]() {
    size_t o = 0;
    for (const Keep& k : keep) {
      cudaMemcpyAsync(k.buf, saved + o, k.bytes, cudaMemcpyDeviceToDevice, h->stream);
      o += k.bytes;
    }
    cudaFreeAsync(saved, h->stream);
  };
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int nt : cand) {
    if (!shape_fits(h, nt)) continue;
    if ((nt & S) && ensure_split(h) != BT_OK) continue;   // no room for the deposit rows
    // the flux step reads f and writes the other buffer (and the moments,
    // and the split form's deposit rows), so repeated launches leave the
    // state unchanged
    auto run = [&]() {
      int r = bt::launch_flux_collide(h->tb, h->st, dt, h->mixed, nt, h->dep, h->rec, h->stream);
      if (!r && (nt & S)) r = bt::launch_zone_collide(h->tb, h->st, dt, h->mixed, h->dep, h->rec, h->stream);
      return r;
    };
    int e = run();
    if (e) { restore(); cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail((cudaError_t)e, "autotune"); }
    cudaEventRecord(a, h->stream);
    for (int k = 0; k < 3; ++k) run();
    cudaEventRecord(b, h->stream);
    cudaError_t ce = cudaEventSynchronize(b);
    float ms = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, a, b);
    if (ce != cudaSuccess) { restore(); cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(ce, "autotune timing"); }
    h->launches += 4;
    if (best == 0.f || ms < best) { best = ms; best_nt = nt; }
  }
  restore();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->nt = best_nt;
  if (!(best_nt & S)) release_split(h);
  tune_store(h->tune_key, best_nt);
  if (chosen_nt) *chosen_nt = best_nt;
  return check_flag(h);
}

int bt_launch_shape(const bt_handle* h, int* threads_per_cta) {
  if (!h || !threads_per_cta) return fail(BT_ERR_ARG, "NULL");
  *threads_per_cta = h->nt;
  return BT_OK;
}

int bt_set_launch_shape(bt_handle* h, int threads_per_cta) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (!valid_shape(threads_per_cta))
    return fail(BT_ERR_ARG, "launch shape must be 128, 256, 512, or BT_SHAPE_SPLIT | 256, 384 or 512");
  if (!shape_fits(h, threads_per_cta)) return fail(BT_ERR_ARG, "launch shape does not fit this problem");
  if (threads_per_cta & bt::kShapeSplit) {
    int rc = ensure_split(h);
    if (rc != BT_OK) return rc;
  } else {
    release_split(h);
  }
  h->nt = threads_per_cta;
  return BT_OK;
}

int bt_moments(bt_handle* h, int mem, double* dN, double* dE, double* dP, double* Q_Ye) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  const size_t n = (size_t)h->cfg.n_species * h->nzone;
  auto kind = mem == BT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (dN && e == cudaSuccess) e = cudaMemcpyAsync(dN, h->st.mom_N, 8 * n, kind, h->stream);
  if (dE && e == cudaSuccess) e = cudaMemcpyAsync(dE, h->st.mom_E, 8 * n, kind, h->stream);
  if (dP && e == cudaSuccess) e = cudaMemcpyAsync(dP, h->st.mom_P, 8 * 3 * n, kind, h->stream);
  if (Q_Ye && e == cudaSuccess) e = cudaMemcpyAsync(Q_Ye, h->qye, 8 * h->nzone, kind, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_moments");
  return check_flag(h);
}

int bt_totals(bt_handle* h, double* N, double* E, double* N_out, double* E_out) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (!h->has_bg) return fail(BT_ERR_STATE, "bt_totals before bt_set_background");
  bind_state(h);
  const int ns = h->cfg.n_species;
  int e = bt::launch_totals(h->tb, h->st, h->mixed, h->tmp, h->stream);
  h->launches += 2;
  if (e) return cuda_fail((cudaError_t)e, "totals");
  std::vector<double> t(2 * ns), acc(4 * ns);
  cudaError_t ce = cudaMemcpyAsync(t.data(), h->tmp, 8 * 2 * ns, cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(acc.data(), h->st.acc, 8 * 4 * ns, cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_totals");
  for (int s = 0; s < ns; ++s) {
    if (N) N[s] = t[2 * s];
    if (E) E[s] = t[2 * s + 1];
    if (N_out) N_out[s] = acc[2 * (2 * s)] + acc[2 * (2 * s) + 1];
    if (E_out) E_out[s] = acc[2 * (2 * s + 1)] + acc[2 * (2 * s + 1) + 1];
  }
  return check_flag(h);
}

int bt_jhk(bt_handle* h, int mem, double* J, double* H, double* K) {
  if (!h || !J || !H || !K) return fail(BT_ERR_ARG, "NULL");
  bind_state(h);
  const size_t n = (size_t)h->cfg.n_species * h->nzone * h->cfg.n_eps;
  double* d = nullptr;
  bool tmp = mem != BT_MEM_DEVICE;
  if (tmp) {
    cudaError_t ce = cudaMallocAsync(&d, 3 * 8 * n, h->stream);
    if (ce != cudaSuccess) return cuda_fail(ce, "bt_jhk alloc");
  }
  double* dJ = tmp ? d : J;
  double* dH = tmp ? d + n : H;
  double* dK = tmp ? d + 2 * n : K;
  int e = bt::launch_jhk(h->tb, h->st, h->mixed, dJ, dH, dK, h->stream);
  h->launches += 1;
  if (e) return cuda_fail((cudaError_t)e, "jhk");
  if (tmp) {
    cudaMemcpyAsync(J, dJ, 8 * n, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(H, dH, 8 * n, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(K, dK, 8 * n, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d, h->stream);
  }
  cudaError_t ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_jhk");
  return BT_OK;
}

int64_t bt_launch_count(const bt_handle* h) { return h ? h->launches : 0; }

int bt_set_surrogate(bt_handle* h, bt_surrogate* s, double tol) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  if (s && !h->mixed) return fail(BT_ERR_ARG, "the learned remap runs in the mixed-precision path only");
  if (s && !(tol >= 0.0) ) return fail(BT_ERR_ARG, "tol must be >= 0");
  if (s && s->stream != h->stream) return fail(BT_ERR_ARG, "network and handle must share a stream");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_set_surrogate");
  if (s && !h->sur_tab) {
    e = cudaMalloc(&h->sur_tab, bt::sur_table_bytes(h->tb));
    if (e == cudaSuccess) e = cudaMalloc(&h->sur_counts, 16);
    if (e == cudaSuccess) e = cudaMemset(h->sur_counts, 0, 16);
    if (e != cudaSuccess) {
      if (h->sur_tab) cudaFree(h->sur_tab);
      h->sur_tab = nullptr;
      return cuda_fail(e, "learned remap table");
    }
  }
  ++h->gen;
  h->sur = s;
  h->sur_tol = (float)tol;
  return BT_OK;
}

int bt_sur_stats(bt_handle* h, int64_t* n_eval, int64_t* n_trip) {
  if (!h || !n_eval || !n_trip) return fail(BT_ERR_ARG, "NULL");
  unsigned long long c[2] = {0, 0};
  if (h->sur_counts) {
    cudaError_t e = cudaMemcpyAsync(c, h->sur_counts, 16, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bt_sur_stats");
  }
  *n_eval = (int64_t)c[0];
  *n_trip = (int64_t)c[1];
  return check_flag(h);
}

int bt_sur_samples(bt_handle* h, const int32_t* idx, int64_t n, float* X, float* Y, int32_t* valid) {
  if (!h || (n > 0 && (!idx || !X || !Y || !valid)) || n < 0) return fail(BT_ERR_ARG, "NULL or n < 0");
  if (h->n_bg < 2) return fail(BT_ERR_STATE, "bt_sur_samples needs a previous and a current background");
  bind_state(h);
  int e = bt::launch_sur_samples(h->tb, h->st, idx, (long long)n, X, Y, valid, h->stream);
  h->launches += n > 0 ? 1 : 0;
  if (e) return cuda_fail((cudaError_t)e, "bt_sur_samples");
  cudaError_t ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "bt_sur_samples");
  return BT_OK;
}

// ---------------------------------------------------------------------------
// Batched step: many independent problems advanced by one graph launch.
// ---------------------------------------------------------------------------
struct bt_batch {
  std::vector<bt_handle*> m;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> side;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::map<std::vector<double>, cudaGraphExec_t> graphs;
  int64_t graph_launches = 0;
};

int bt_batch_destroy(bt_batch* b) {
  if (!b) return BT_OK;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaStream_t st : b->side) cudaStreamDestroy(st);
  for (bt_handle* h : b->m) bt_destroy(h);
  delete b;
  return BT_OK;
}

int bt_batch_create(const bt_config* cfgs, int n, void* stream, bt_batch** out) {
  if (!cfgs || n < 1 || !out) return fail(BT_ERR_ARG, "cfgs/n/out");
  if (!stream) return fail(BT_ERR_ARG, "the batch needs a created stream (graph capture)");
  *out = nullptr;
  bt_batch* b = new bt_batch();
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    bt_config c = cfgs[i];
    c.stream = stream;
    bt_handle* h = nullptr;
    int rc = bt_create(&c, nullptr, &h);
    if (rc != BT_OK) { bt_batch_destroy(b); return rc; }
    b->m.push_back(h);
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) { bt_batch_destroy(b); return cuda_fail(e, "batch stream"); }
    b->side.push_back(st);
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { bt_batch_destroy(b); return cuda_fail(e, "batch event"); }
    b->join.push_back(ev);
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) { bt_batch_destroy(b); return cuda_fail(e, "batch event"); }
  *out = b;
  return BT_OK;
}

int bt_batch_member(bt_batch* b, int i, bt_handle** out) {
  if (!b || !out || i < 0 || i >= (int)b->m.size()) return fail(BT_ERR_ARG, "member index");
  *out = b->m[i];
  return BT_OK;
}

int bt_batch_step(bt_batch* b, const double* dt) {
  if (!b || !dt) return fail(BT_ERR_ARG, "NULL");
  const int n = (int)b->m.size();
  std::vector<double> key;
  for (int i = 0; i < n; ++i) {
    bt_handle* h = b->m[i];
    if (!h->has_bg) return fail(BT_ERR_STATE, "batch member without a background");
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) return fail(BT_ERR_DT, "dt must be positive and finite");
    key.push_back(h->cur);
    key.push_back(h->fcur);
    key.push_back(h->remap_pending ? 1 : 0);
    key.push_back(dt[i]);
    key.push_back(h->nt);
    key.push_back(h->sur ? 1.0 : 0.0);
    key.push_back(h->sur_tol);
    key.push_back((double)h->gen);   // the buffers the graph would read
  }
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    if (b->graphs.size() >= 16) {
      for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
      b->graphs.clear();
    }
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    cudaEventRecord(b->fork, b->stream);
    int rc = BT_OK;
    for (int i = 0; i < n && rc == BT_OK; ++i) {
      bt_handle* h = b->m[i];
      cudaStreamWaitEvent(b->side[i], b->fork, 0);
      cudaStream_t saved = h->stream;
      const bool prof = h->prof, pend = h->remap_pending;
      const int fcur = h->fcur;
      const int64_t launches = h->launches;
      h->stream = b->side[i];
      h->prof = false;
      rc = step_enqueue(h, dt[i]);
      // capture records the work; the state advances when the graph runs
      h->stream = saved; h->prof = prof; h->remap_pending = pend; h->fcur = fcur; h->launches = launches;
      cudaEventRecord(b->join[i], b->side[i]);
      cudaStreamWaitEvent(b->stream, b->join[i], 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->stream, &graph);
    if (rc != BT_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    it = b->graphs.emplace(key, exec).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second, b->stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  b->graph_launches += 1;
  for (bt_handle* h : b->m) {
    h->launches += (h->remap_pending ? 1 : 0) + (h->sur ? 1 : 0) + ((h->nt & bt::kShapeSplit) ? 1 : 0) + 3;
    h->remap_pending = false;
    h->fcur = 1 - h->fcur;
  }
  return BT_OK;
}

int64_t bt_batch_launch_count(const bt_batch* b) {
  if (!b) return 0;
  int64_t n = 0;
  for (const bt_handle* h : b->m) n += h->launches;
  return n;
}

int64_t bt_batch_graph_launches(const bt_batch* b) { return b ? b->graph_launches : 0; }

int bt_profile(bt_handle* h, int enable) {
  if (!h) return fail(BT_ERR_ARG, "NULL");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_profile");
  prof_clear(h);
  h->prof = enable != 0;
  return BT_OK;
}

int bt_profile_read(bt_handle* h, int kernel, double* total_ms, int64_t* launches) {
  if (!h || !total_ms || !launches) return fail(BT_ERR_ARG, "NULL");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_profile_read");
  double tot = 0.0;
  int64_t n = 0;
  for (size_t i = 0; i < h->prof_id.size(); ++i) {
    if (h->prof_id[i] != kernel) continue;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    tot += ms;
    ++n;
  }
  *total_ms = tot;
  *launches = n;
  return BT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The learned remap's network (bt_sur_*): parameters, normaliser, Adam state.
// ---------------------------------------------------------------------------

namespace {

std::mutex g_mlp_mutex;
bool g_mlp_prepared[64];

int sur_sync(bt_surrogate* s, const char* what) {
  int fl[4];
  cudaError_t e = cudaMemcpyAsync(fl, s->flag, 16, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (fl[1]) return fail(BT_ERR_TIMEOUT, std::string(what) + ": a tensor-core wait gave up");
  return BT_OK;
}

}  // namespace

extern "C" {

int bt_sur_create(void* stream, bt_surrogate** out) {
  if (!out) return fail(BT_ERR_ARG, "NULL");
  *out = nullptr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  {
    std::lock_guard<std::mutex> lock(g_mlp_mutex);
    if (dev >= 0 && dev < 64 && !g_mlp_prepared[dev]) {
      int rc = bt::mlp::prepare();
      if (rc) return cuda_fail((cudaError_t)rc, "network kernels: shared memory opt-in");
      g_mlp_prepared[dev] = true;
    }
  }
  bt_surrogate* s = new bt_surrogate();
  s->stream = (cudaStream_t)stream;
  cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const size_t np = bt::mlp::kNParam, nt = bt::mlp::kNTrain;
  e = cudaMalloc(&s->prm, 4 * np);
  if (e == cudaSuccess) e = cudaMalloc(&s->grad, 4 * np);
  if (e == cudaSuccess) e = cudaMalloc(&s->m, 4 * nt);
  if (e == cudaSuccess) e = cudaMalloc(&s->v, 4 * nt);
  if (e == cudaSuccess) e = cudaMalloc(&s->loss, 4 * 8);
  if (e == cudaSuccess) e = cudaMalloc(&s->flag, 16);
  if (e == cudaSuccess) e = cudaMalloc(&s->stats, 8 * 32);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->prm, 0, 4 * np, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->m, 0, 4 * nt, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->v, 0, 4 * nt, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->flag, 0, 16, s->stream);
  if (e == cudaSuccess) {
    // identity normaliser until bt_sur_fit_normalizer or bt_sur_set_params
    std::vector<float> one(bt::mlp::kIn, 1.0f);
    e = cudaMemcpyAsync(s->prm + bt::mlp::oScale, one.data(), 4 * bt::mlp::kIn, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  if (e != cudaSuccess) {
    bt_sur_destroy(s);
    return cuda_fail(e, "bt_sur_create");
  }
  *out = s;
  return BT_OK;
}

int bt_sur_destroy(bt_surrogate* s) {
  if (!s) return BT_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->prm);
  cudaFree(s->grad);
  cudaFree(s->m);
  cudaFree(s->v);
  cudaFree(s->loss);
  cudaFree(s->flag);
  cudaFree(s->stats);
  delete s;
  return BT_OK;
}

int bt_sur_set_params(bt_surrogate* s, int mem, const float* p) {
  if (!s || !p) return fail(BT_ERR_ARG, "NULL");
  cudaError_t e = cudaMemcpyAsync(s->prm, p, 4 * (size_t)bt::mlp::kNParam,
                                  mem == BT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->m, 0, 4 * (size_t)bt::mlp::kNTrain, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->v, 0, 4 * (size_t)bt::mlp::kNTrain, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_set_params");
  s->adam_t = 0;
  return BT_OK;
}

int bt_sur_get_params(bt_surrogate* s, int mem, float* p) {
  if (!s || !p) return fail(BT_ERR_ARG, "NULL");
  cudaError_t e = cudaMemcpyAsync(p, s->prm, 4 * (size_t)bt::mlp::kNParam,
                                  mem == BT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_get_params");
  return BT_OK;
}

int bt_sur_fit_normalizer(bt_surrogate* s, const float* X, int64_t n) {
  if (!s || !X || n < 2) return fail(BT_ERR_ARG, "NULL or n < 2");
  cudaError_t e = cudaMemsetAsync(s->stats, 0, 8 * 32, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_fit_normalizer");
  int rc = bt::mlp::launch_feat_stats(X, n, s->stats, s->stream);
  if (rc) return cuda_fail((cudaError_t)rc, "feature statistics");
  double acc[32];
  e = cudaMemcpyAsync(acc, s->stats, 8 * 32, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_fit_normalizer");
  float ms[32];
  for (int i = 0; i < 16; ++i) {
    const double mean = acc[i] / (double)n;
    const double var = std::max(acc[16 + i] / (double)n - mean * mean, 0.0);
    const double sd = std::sqrt(var);
    ms[i] = (float)mean;
    ms[16 + i] = (float)(sd > 1e-12 * (1.0 + std::fabs(mean)) ? 1.0 / sd : 1.0);
  }
  e = cudaMemcpyAsync(s->prm + bt::mlp::oMean, ms, 4 * 32, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_fit_normalizer");
  return BT_OK;
}

int bt_sur_forward(bt_surrogate* s, const float* X, int64_t n, float* P) {
  if (!s || (n > 0 && (!X || !P)) || n < 0) return fail(BT_ERR_ARG, "NULL or n < 0");
  int rc = bt::mlp::launch_forward(s->prm, X, n, P, s->flag, 4 * s->n_sm, s->stream);
  if (rc) return cuda_fail((cudaError_t)rc, "network forward");
  return sur_sync(s, "bt_sur_forward");
}

int bt_sur_grad(bt_surrogate* s, const float* X, const float* Y, int64_t n, float* grad, float* loss) {
  if (!s || !X || !Y || !grad || !loss || n < 1) return fail(BT_ERR_ARG, "NULL or n < 1");
  cudaError_t e = cudaMemsetAsync(grad, 0, 4 * (size_t)bt::mlp::kNParam, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, 4, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_grad");
  int rc = bt::mlp::launch_grad(s->prm, X, Y, n, 1.0f / (float)n, grad, loss, s->flag, s->n_sm, s->stream);
  if (rc) return cuda_fail((cudaError_t)rc, "network gradient");
  return sur_sync(s, "bt_sur_grad");
}

int bt_sur_train(bt_surrogate* s, const float* X, const float* Y, int64_t n, const bt_train_cfg* cfg,
                 float* loss_log) {
  if (!s || !X || !Y || !cfg || n < 1) return fail(BT_ERR_ARG, "NULL or n < 1");
  if (cfg->epochs < 1 || cfg->batch < 1) return fail(BT_ERR_ARG, "epochs and batch must be >= 1");
  const int64_t batch = std::min<int64_t>(cfg->batch, n);
  const int64_t steps = (n + batch - 1) / batch;
  const int64_t total = steps * cfg->epochs;
  float* eloss = nullptr;
  cudaError_t e = cudaMallocAsync(&eloss, 4 * (size_t)cfg->epochs, s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(eloss, 0, 4 * (size_t)cfg->epochs, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_train");
  int64_t k = 0;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    for (int64_t b = 0; b < steps; ++b, ++k) {
      const int64_t b0 = b * batch, nb = std::min(batch, n - b0);
      e = cudaMemsetAsync(s->grad, 0, 4 * (size_t)bt::mlp::kNParam, s->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->loss, 0, 4, s->stream);
      if (e != cudaSuccess) { cudaFreeAsync(eloss, s->stream); return cuda_fail(e, "bt_sur_train"); }
      int rc = bt::mlp::launch_grad(s->prm, X + b0 * bt::mlp::kIn, Y + b0 * bt::mlp::kOut, nb, 1.0f / (float)nb,
                                    s->grad, s->loss, s->flag, s->n_sm, s->stream);
      // cosine decay from lr to lr_final over the run
      const double c = 0.5 * (1.0 + std::cos(kPi * (double)k / (double)std::max<int64_t>(total - 1, 1)));
      const float lr = (float)(cfg->lr_final + (cfg->lr - cfg->lr_final) * c);
      ++s->adam_t;
      const float bc1 = (float)(1.0 - std::pow((double)cfg->beta1, (double)s->adam_t));
      const float bc2 = (float)(1.0 - std::pow((double)cfg->beta2, (double)s->adam_t));
      if (!rc)
        rc = bt::mlp::launch_adam(s->prm, s->grad, s->m, s->v, lr, cfg->beta1, cfg->beta2, cfg->eps, bc1, bc2,
                                  s->loss, eloss + ep, s->stream);
      if (rc) { cudaFreeAsync(eloss, s->stream); return cuda_fail((cudaError_t)rc, "network training"); }
    }
  }
  std::vector<float> lg(cfg->epochs);
  e = cudaMemcpyAsync(lg.data(), eloss, 4 * (size_t)cfg->epochs, cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(eloss, s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "bt_sur_train");
  int rc = sur_sync(s, "bt_sur_train");
  if (rc != BT_OK) return rc;
  if (loss_log)
    for (int ep = 0; ep < cfg->epochs; ++ep) loss_log[ep] = lg[ep] / (float)steps;
  return BT_OK;
}

}  // extern "C"
