/*
 * bt_oracle.c -- plain, slow, FP64 CPU oracle of one transport step of the
 * discrete-ordinate Boltzmann scheme of Chan & Mueller (arXiv:2003.02845).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library
 * shares no code with it (no headers, helpers, tables or constants).
 *
 * Every routine follows the paper's definitions in the paper's order and is
 * written for a reader checking it against the paper by eye: loops over
 * species, zones, faces, groups and angles; the remap operator T is applied
 * bin by bin as an explicit deposit into eight destination bins.  Readings of
 * points the paper leaves open are tagged [R-n]; the same numbers label the
 * readings listed in the design notes.
 *
 * Units: c = 1.  f layout: f[s][zone][group][angle], zone = b*n_r + a,
 * angle = j*n_phi + k (mu index j, Phi index k).
 *
 * Parity: every function is pinned by the CPU test-suite against closed
 * forms, textbook special cases or brute force (see tests/test_oracle_*.py).
 *
 * Threads (OpenMP, when built with it): the faces of a step are taken in
 * blocks; within a block every face's flux and its two remapped deposits
 * are computed in parallel into buffers of their own, then added to the
 * zones' content changes one face after another in face-list order.  The
 * time remap and the collision solve are independent per zone.  Results are
 * therefore the same bit for bit for any number of threads.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_ 3.14159265358979323846

enum { ORC_SPHERICAL = 0, ORC_SLAB = 1 };
enum { KICK_R = 0, KICK_TH = 1, KICK_PH = 2, KICK_TIME = 3, KICK_NONE = 4 };

/* ------------------------------------------------------------------------- */
/* Small vector helpers                                                      */
/* ------------------------------------------------------------------------- */
static double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double *a, const double *b, double *c) {
  c[0] = a[1]*b[2] - a[2]*b[1];
  c[1] = a[2]*b[0] - a[0]*b[2];
  c[2] = a[0]*b[1] - a[1]*b[0];
}

/* ------------------------------------------------------------------------- */
/* Momentum grid (Sec. 3.1)                                                  */
/* ------------------------------------------------------------------------- */
/* Legendre polynomial P_n(x) and its derivative by the three-term recurrence. */
static void legendre(int n, double x, double *p, double *dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0*k - 1.0)*x*p1 - (k - 1.0)*p0) / k;
    p0 = p1; p1 = p2;
  }
  *p = p1;
  *dp = n * (x*p1 - p0) / (x*x - 1.0);
}

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1] by Newton's
 * method; nodes are made exactly antisymmetric, weights exactly symmetric.
 * [R-2] the mu cells are the Gauss-Legendre cells: node mu_j is the cell's
 * direction, its weight the cell width (Sec. 3.1, widths = quadrature weights). */
void orc_gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(PI_ * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, &p, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, &p, &dp);
    double wi = 2.0 / ((1.0 - z*z) * dp * dp);
    /* i-th largest node */
    x[n - 1 - i] = z;  x[i] = -z;
    w[n - 1 - i] = wi; w[i] = wi;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

/* Gauss-Lobatto nodes (ascending, x[0] = -1, x[n-1] = 1) and weights on
 * [-1, 1], n >= 2: the interior nodes are the roots of P'_{n-1}, found by
 * Newton's method on P'_{n-1} from the Chebyshev-Lobatto points, and
 * w_i = 2 / (n (n-1) P_{n-1}(x_i)^2).
 * [R-2] Sec. 3.1 asks for mu cells whose widths are the Gauss-Lobatto weights:
 * node mu_j is the cell's direction (mu = +-1 among them), its weight the
 * cell's width. */
void orc_gauss_lobatto(int n, double *x, double *w) {
  int N = n - 1;   /* degree of the Legendre polynomial */
  x[0] = -1.0; x[N] = 1.0;
  w[0] = w[N] = 2.0 / (n * (double)N);
  for (int i = 1; i <= N / 2; ++i) {
    /* i-th largest interior root of P'_N */
    double z = cos(PI_ * i / N);
    for (int it = 0; it < 100; ++it) {
      /* P'_N and P''_N from P_N, P_{N-1}: (1-z^2) P'' = 2 z P' - N (N+1) P */
      double p, dp;
      legendre(N, z, &p, &dp);
      double d2p = (2.0*z*dp - N*(N + 1.0)*p) / (1.0 - z*z);
      double dz = dp / d2p;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(N, z, &p, &dp);
    double wi = 2.0 / (n * (double)N * p * p);
    x[N - i] = z;  x[i] = -z;
    w[N - i] = wi; w[i] = wi;
  }
  if (n % 2 == 1) {   /* odd n: the centre node */
    double p, dp;
    legendre(N, 0.0, &p, &dp);
    x[N / 2] = 0.0;
    w[N / 2] = 2.0 / (n * (double)N * p * p);
  }
}

/* ------------------------------------------------------------------------- */
/* Frames (Sec. 3.2.1): local orthonormal triad at colatitude th, azimuth ph  */
/* E columns = (r_hat, theta_hat, phi_hat) in Cartesian components.          */
/* ------------------------------------------------------------------------- */
void orc_triad(double th, double ph, double *E /* 3x3 row-major, E[3*m+c] */) {
  double st = sin(th), ct = cos(th), sp = sin(ph), cp = cos(ph);
  double rh[3] = {st*cp, st*sp, ct};
  double thh[3] = {ct*cp, ct*sp, -st};
  double phh[3] = {-sp, cp, 0.0};
  for (int m = 0; m < 3; ++m) { E[3*m+0] = rh[m]; E[3*m+1] = thh[m]; E[3*m+2] = phh[m]; }
}

/* [R-8] G = E_dst^T E_src: components of a vector given in the source triad,
 * expressed in the destination triad (the rotation of Sec. 3.2.1 written as
 * a change of orthonormal basis). */
void orc_rotation(double th_s, double ph_s, double th_d, double ph_d, double *G) {
  double Es[9], Ed[9];
  orc_triad(th_s, ph_s, Es);
  orc_triad(th_d, ph_d, Ed);
  for (int m = 0; m < 3; ++m)
    for (int n = 0; n < 3; ++n) {
      double s = 0.0;
      for (int c = 0; c < 3; ++c) s += Ed[3*c+m] * Es[3*c+n];
      G[3*m+n] = s;
    }
}

/* ------------------------------------------------------------------------- */
/* Lorentz boost Lambda (Sec. 3.2.2) acting on (u0, u1, u2, u3); sign = +1   */
/* comoving -> Eulerian with fluid velocity v, sign = -1 the inverse.        */
/* ------------------------------------------------------------------------- */
void orc_boost(const double *v_in, int sign, const double *u, double *out) {
  double v[3] = {sign * v_in[0], sign * v_in[1], sign * v_in[2]};
  double v2 = dot3(v, v);
  double g = 1.0 / sqrt(1.0 - v2);
  double L[4][4];
  L[0][0] = g;
  for (int i = 0; i < 3; ++i) { L[0][i+1] = g*v[i]; L[i+1][0] = g*v[i]; }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      /* (gamma-1) v_i v_j / v^2, with (gamma-1)/v^2 = gamma^2/(gamma+1) */
      double c = (g*g/(g + 1.0)) * v[i]*v[j];
      L[i+1][j+1] = (i == j ? 1.0 : 0.0) + c;
    }
  for (int m = 0; m < 4; ++m) {
    double s = 0.0;
    for (int n = 0; n < 4; ++n) s += L[m][n] * u[n];
    out[m] = s;
  }
}

/* ------------------------------------------------------------------------- */
/* Hamiltonian kick K (Sec. 3.2.4) for the CFC metric with zero shift, in    */
/* the Eulerian orthonormal components (e, p) of the source frame.           */
/* Covariant components: u_0 = -alpha e, u_i = phi^2 p_i.                   */
/* Spatial step along axis n: u_0 and the tangential u_i are conserved; the  */
/* normal component follows from the null condition in the destination      */
/* metric, with the root chosen so that delta -> 0 as delta g -> 0; if no    */
/* real root exists the normal covariant component is set to zero and the   */
/* tangential ones are rescaled to restore the null condition ("total        */
/* internal reflection").  [R-16]                                            */
/* Time step (metric changing in time at fixed position): the spatial        */
/* covariant components are conserved and u_0 follows from the null         */
/* condition.  [R-16b]                                                       */
/* Returns 1 if the reflection branch was taken.                             */
/* ------------------------------------------------------------------------- */
int orc_kick(int axis, double a_src, double p_src, double a_dst, double p_dst,
             const double *in /* e,p0,p1,p2 */, double *out) {
  double b = (p_src / p_dst) * (p_src / p_dst);   /* (phi_src/phi_dst)^2 */
  if (axis == KICK_NONE) { for (int i = 0; i < 4; ++i) out[i] = in[i]; return 0; }
  if (axis == KICK_TIME) {
    out[0] = b*in[0]; out[1] = b*in[1]; out[2] = b*in[2]; out[3] = b*in[3];
    return 0;
  }
  double a = a_src / a_dst;                       /* alpha_src/alpha_dst */
  double e_new = a * in[0];
  double pt2 = 0.0;
  for (int i = 0; i < 3; ++i) if (i != axis) pt2 += in[1+i]*in[1+i];
  double pn = in[1+axis];
  /* null condition in the destination metric:
   * pn_new^2 = e_new^2 - b^2 pt^2 = a^2 pn^2 + (a^2 - b^2) pt^2,
   * using e^2 = pn^2 + pt^2 of the source vector. */
  double rad = a*a*pn*pn + (a*a - b*b)*pt2;
  out[0] = e_new;
  if (rad >= 0.0) {
    double s = (pn >= 0.0) ? 1.0 : -1.0;
    for (int i = 0; i < 3; ++i) out[1+i] = b*in[1+i];
    out[1+axis] = s * sqrt(rad);
    return 0;
  }
  /* reflection branch: normal covariant component -> 0, tangential scaled */
  double sc = e_new / sqrt(pt2);
  for (int i = 0; i < 3; ++i) out[1+i] = sc*in[1+i];
  out[1+axis] = 0.0;
  return 1;
}

/* ------------------------------------------------------------------------- */
/* Transformation chain (Sec. 2.2, Sec. 3.2):                                */
/*   u~_dst = Lambda_dst^-1 M_dst^-1 G K(M_src Lambda_src u~_src)            */
/* with the comoving source vector (1, n).  M (Sec. 3.2.3) with zero shift   */
/* only rescales components (u^0 = e/alpha, u^i = p_i/phi^2); it is folded   */
/* into the kick, which is written in Eulerian components.                   */
/* Output: rho = e~_dst (ratio of destination to source comoving energy),   */
/* mu* and Phi* of the destination comoving direction.                       */
/* ------------------------------------------------------------------------- */
int orc_chain(const double *v_src, double a_src, double p_src,
              const double *v_dst, double a_dst, double p_dst,
              const double *G, int axis, const double *n,
              double *rho, double *mu_s, double *Phi_s) {
  double u[4] = {1.0, n[0], n[1], n[2]}, ue[4], uk[4], ur[4], ud[4];
  orc_boost(v_src, +1, u, ue);
  int tir = orc_kick(axis, a_src, p_src, a_dst, p_dst, ue, uk);
  ur[0] = uk[0];
  for (int m = 0; m < 3; ++m) ur[1+m] = G[3*m+0]*uk[1] + G[3*m+1]*uk[2] + G[3*m+2]*uk[3];
  orc_boost(v_dst, -1, ur, ud);
  *rho = ud[0];
  double mu = ud[1] / ud[0];
  if (mu > 1.0) mu = 1.0;
  if (mu < -1.0) mu = -1.0;
  *mu_s = mu;
  double ph = atan2(ud[3], ud[2]);
  if (ph < 0.0) ph += 2.0*PI_;
  *Phi_s = ph;
  return tir;
}

/* ------------------------------------------------------------------------- */
/* Interpolation weights (Sec. 3.2, number, direction and energy conserved   */
/* by linear weights per axis).  Each returns the left index and the right   */
/* weight; the left weight is 1 - w.                                         */
/* ------------------------------------------------------------------------- */
/* [R-4] energy: centres have the constant ratio R; target eps* = rho eps_i;
 * bracket eps_{i+m} <= eps* < eps_{i+m+1}; w linear in eps.  [R-7] targets
 * outside the group range are clamped to the extreme group. */
void orc_weights_eps(double rho, double R, int *m, double *w) {
  int mm = (int)floor(log(rho) / log(R));
  double t = rho / pow(R, (double)mm);
  double ww = (t - 1.0) / (R - 1.0);
  if (ww < 0.0) ww = 0.0;
  if (ww > 1.0) ww = 1.0;
  *m = mm; *w = ww;
}

/* mu: linear between the bracketing nodes; outside [mu_0, mu_{N-1}] all
 * weight goes to the extreme node [R-7]. */
void orc_weights_mu(double mus, int n_mu, const double *mu, int *jL, double *w) {
  if (n_mu == 1) { *jL = 0; *w = 0.0; return; }
  if (mus <= mu[0]) { *jL = 0; *w = 0.0; return; }
  if (mus >= mu[n_mu-1]) { *jL = n_mu - 2; *w = 1.0; return; }
  int j = 0;
  while (j < n_mu - 2 && mu[j+1] <= mus) ++j;
  *jL = j;
  *w = (mus - mu[j]) / (mu[j+1] - mu[j]);
}

/* [R-6] Phi: linear in Phi between the bracketing centres with periodic wrap. */
void orc_weights_phi(double Phis, int n_phi, int *kL, double *w) {
  if (n_phi == 1) { *kL = 0; *w = 0.0; return; }
  double dP = 2.0*PI_ / n_phi;
  double u = Phis / dP - 0.5;
  double k = floor(u);
  double ww = u - k;
  int kk = (int)k % n_phi;
  if (kk < 0) kk += n_phi;
  *kL = kk; *w = ww;
}

/* ------------------------------------------------------------------------- */
/* Implicit collision solve (Sec. 3.5) for one (zone, group):                */
/*   (1 + (ka+ks) tau_b) f_b - ks tau_b J = r_b,  J = (1/4pi) sum dOm_b f_b  */
/* [R-9] exact Sherman-Morrison solution of the backward-Euler system.       */
/* ------------------------------------------------------------------------- */
void orc_collision_row(int n_ang, const double *r, const double *tau, double ka, double ks,
                       const double *dOm, double *f) {
  double Sr = 0.0, S1 = 0.0;
  for (int b = 0; b < n_ang; ++b) {
    double D = 1.0 + (ka + ks) * tau[b];
    Sr += dOm[b] * r[b] / D;
    S1 += dOm[b] * (1.0 + ka * tau[b]) / D;
  }
  double J = Sr / S1;
  for (int b = 0; b < n_ang; ++b) {
    double D = 1.0 + (ka + ks) * tau[b];
    f[b] = (r[b] + ks * tau[b] * J) / D;
  }
}

/* MC limiter (van Leer 1977) on two one-sided slopes. */
static double mc_limiter(double a, double b) {
  if (a * b <= 0.0) return 0.0;
  double s = a > 0.0 ? 1.0 : -1.0;
  double x = fabs(2.0*a), y = fabs(2.0*b), z = 0.5*fabs(a + b);
  double m = x < y ? x : y;
  m = m < z ? m : z;
  return s * m;
}
double orc_mc(double a, double b) { return mc_limiter(a, b); }

/* ------------------------------------------------------------------------- */
/* Geometry (Sec. 3.1): flat-faced cells bounded by the vertices of the      */
/* spherical-polar grid.                                                     */
/* ------------------------------------------------------------------------- */
static void vertex(double r, double th, double ph, double *x) {
  x[0] = r*sin(th)*cos(ph); x[1] = r*sin(th)*sin(ph); x[2] = r*cos(th);
}
/* area of the planar quadrilateral v0 v1 v2 v3 (vertices in cyclic order) */
static double quad_area(const double *v0, const double *v1, const double *v2, const double *v3) {
  double d1[3], d2[3], c[3];
  for (int i = 0; i < 3; ++i) { d1[i] = v2[i] - v0[i]; d2[i] = v3[i] - v1[i]; }
  cross3(d1, d2, c);
  return 0.5 * sqrt(dot3(c, c));
}
double orc_face_area_r(double r, double th0, double th1, double dphi) {
  double a[3], b[3], c[3], d[3];
  vertex(r, th0, -0.5*dphi, a); vertex(r, th0, 0.5*dphi, b);
  vertex(r, th1, 0.5*dphi, c);  vertex(r, th1, -0.5*dphi, d);
  return quad_area(a, b, c, d);
}
double orc_face_area_th(double r0, double r1, double th, double dphi) {
  double a[3], b[3], c[3], d[3];
  vertex(r0, th, -0.5*dphi, a); vertex(r0, th, 0.5*dphi, b);
  vertex(r1, th, 0.5*dphi, c);  vertex(r1, th, -0.5*dphi, d);
  return quad_area(a, b, c, d);
}
double orc_face_area_ph(double r0, double r1, double th0, double th1, double ph) {
  double a[3], b[3], c[3], d[3];
  vertex(r0, th0, ph, a); vertex(r0, th1, ph, b);
  vertex(r1, th1, ph, c); vertex(r1, th0, ph, d);
  return quad_area(a, b, c, d);
}
/* volume of the convex hexahedron: sum of tetrahedra from the vertex
 * centroid to two triangles of each face */
static double tet_vol(const double *a, const double *b, const double *c, const double *o) {
  double x[3], y[3], z[3], cr[3];
  for (int i = 0; i < 3; ++i) { x[i] = a[i]-o[i]; y[i] = b[i]-o[i]; z[i] = c[i]-o[i]; }
  cross3(y, z, cr);
  return fabs(dot3(x, cr)) / 6.0;
}
double orc_cell_volume(double r0, double r1, double th0, double th1, double dphi) {
  double V[8][3];
  int idx = 0;
  for (int ir = 0; ir < 2; ++ir)
    for (int it = 0; it < 2; ++it)
      for (int ip = 0; ip < 2; ++ip)
        vertex(ir ? r1 : r0, it ? th1 : th0, ip ? 0.5*dphi : -0.5*dphi, V[idx++]);
  double o[3] = {0, 0, 0};
  for (int k = 0; k < 8; ++k) for (int i = 0; i < 3; ++i) o[i] += V[k][i] / 8.0;
  /* faces as vertex index quads: vertex index = 4*ir + 2*it + ip */
  static const int F[6][4] = {
    {0, 1, 3, 2}, {4, 5, 7, 6},   /* r0, r1 */
    {0, 1, 5, 4}, {2, 3, 7, 6},   /* th0, th1 */
    {0, 2, 6, 4}, {1, 3, 7, 5}};  /* ph0, ph1 */
  double vol = 0.0;
  for (int f = 0; f < 6; ++f) {
    vol += tet_vol(V[F[f][0]], V[F[f][1]], V[F[f][2]], o);
    vol += tet_vol(V[F[f][0]], V[F[f][2]], V[F[f][3]], o);
  }
  return vol;
}

/* ------------------------------------------------------------------------- */
/* Problem state                                                             */
/* ------------------------------------------------------------------------- */
typedef struct {
  int geom, n_r, n_th, periodic_th;
  double dth_col, dphi;
  double th_max;               /* 2D polar range [0, th_max]; th_max < pi: open face at th_max */
  double *fbc;                 /* [s][n_r][e] distribution imposed on the incoming bins of the th_max face */
  double *r_e, *th_e;
  int n_s, n_e, n_mu, n_ph, n_ang;
  int lobatto;                 /* [R-2] mu cells on Gauss-Lobatto nodes (pole nodes mu = +-1) */
  int *kind;
  double *e_e, *e_c, *dGam, R;
  double *mu, *dmu, *Phc, *dOm;
  double *vol;                 /* [zone] */
  double *f;                   /* [s][zone][e][ang] */
  double *v, *al, *ph;         /* current background */
  double *v0, *al0, *ph0;      /* previous background (time remap) */
  double *ka, *ks, *fe;        /* [s][zone][e] */
  int has_bg, remap_pending;
  int has_prev;                /* v0, al0, ph0 hold a previous background */
  double phase_norm;
  /* last-step outputs */
  double *dN, *dE, *dP;        /* [s][zone], [s][zone], [s][zone][3] */
  double *N_out, *E_out;       /* [s] cumulative outflow through open boundaries */
  int n_tir;
  /* [R-7] diagnostics: deposits whose energy target lay past the first or
   * last group (clamped into it), and source bins whose mu target lay past
   * the outermost node */
  long n_clamp_e, n_clamp_mu;
} orc_t;

static int nz(const orc_t *o) { return o->n_r * o->n_th; }
static size_t nrow(const orc_t *o) { return (size_t)o->n_e * o->n_ang; }

/* [R-4] group centre = number-weighted mean energy of a bin with constant f:
 * eps_i = 3/4 (e+^4 - e-^4)/(e+^3 - e-^3);  dGamma_i = (e+^3 - e-^3)/3. */
orc_t *orc_create(int geom, int n_r, int n_th, const double *r_edges, int periodic_th,
                  double dth_col, double dphi, int n_s, const int *kind,
                  int n_e, const double *e_edges, int n_mu, int n_ph, double phase_norm, int lobatto,
                  double th_max) {
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  o->th_max = (th_max > 0.0 && !periodic_th && geom == ORC_SPHERICAL) ? th_max : PI_;
  o->fbc = (double *)calloc((size_t)n_s * n_r * n_e, sizeof(double));
  o->lobatto = lobatto && n_mu >= 2;
  o->geom = geom; o->n_r = n_r; o->n_th = n_th; o->periodic_th = periodic_th;
  o->dth_col = dth_col; o->dphi = dphi; o->n_s = n_s; o->n_e = n_e;
  o->n_mu = n_mu; o->n_ph = n_ph; o->n_ang = n_mu * n_ph; o->phase_norm = phase_norm;
  o->r_e = (double *)malloc(sizeof(double) * (n_r + 1));
  memcpy(o->r_e, r_edges, sizeof(double) * (n_r + 1));
  o->th_e = (double *)malloc(sizeof(double) * (n_th + 1));
  if (periodic_th) {
    o->th_e[0] = 0.5*PI_ - 0.5*dth_col; o->th_e[1] = 0.5*PI_ + 0.5*dth_col;
  } else {
    for (int b = 0; b <= n_th; ++b) o->th_e[b] = o->th_max * b / n_th;
  }
  o->kind = (int *)malloc(sizeof(int) * n_s);
  memcpy(o->kind, kind, sizeof(int) * n_s);
  o->e_e = (double *)malloc(sizeof(double) * (n_e + 1));
  memcpy(o->e_e, e_edges, sizeof(double) * (n_e + 1));
  o->e_c = (double *)malloc(sizeof(double) * n_e);
  o->dGam = (double *)malloc(sizeof(double) * n_e);
  for (int i = 0; i < n_e; ++i) {
    double a = e_edges[i], b = e_edges[i+1];
    o->e_c[i] = 0.75 * (pow(b, 4) - pow(a, 4)) / (pow(b, 3) - pow(a, 3));
    o->dGam[i] = (pow(b, 3) - pow(a, 3)) / 3.0;
  }
  o->R = n_e > 1 ? o->e_c[1] / o->e_c[0] : 2.0;
  o->mu = (double *)malloc(sizeof(double) * n_mu);
  o->dmu = (double *)malloc(sizeof(double) * n_mu);
  if (o->lobatto) orc_gauss_lobatto(n_mu, o->mu, o->dmu);
  else orc_gauss_legendre(n_mu, o->mu, o->dmu);
  o->Phc = (double *)malloc(sizeof(double) * n_ph);
  for (int k = 0; k < n_ph; ++k) o->Phc[k] = (k + 0.5) * 2.0*PI_ / n_ph;
  o->dOm = (double *)malloc(sizeof(double) * o->n_ang);
  for (int j = 0; j < n_mu; ++j)
    for (int k = 0; k < n_ph; ++k) o->dOm[j*n_ph + k] = o->dmu[j] * 2.0*PI_ / n_ph;
  int Z = n_r * n_th;
  o->vol = (double *)malloc(sizeof(double) * Z);
  for (int b = 0; b < n_th; ++b)
    for (int a = 0; a < n_r; ++a)
      o->vol[b*n_r + a] = geom == ORC_SLAB ? (r_edges[a+1] - r_edges[a])
          : orc_cell_volume(r_edges[a], r_edges[a+1], o->th_e[b], o->th_e[b+1], dphi);
  size_t N = (size_t)n_s * Z * nrow(o);
  o->f = (double *)calloc(N, sizeof(double));
  o->v = (double *)calloc(3*Z, sizeof(double)); o->v0 = (double *)calloc(3*Z, sizeof(double));
  o->al = (double *)calloc(Z, sizeof(double)); o->al0 = (double *)calloc(Z, sizeof(double));
  o->ph = (double *)calloc(Z, sizeof(double)); o->ph0 = (double *)calloc(Z, sizeof(double));
  size_t NO = (size_t)n_s * Z * n_e;
  o->ka = (double *)calloc(NO, sizeof(double));
  o->ks = (double *)calloc(NO, sizeof(double));
  o->fe = (double *)calloc(NO, sizeof(double));
  o->dN = (double *)calloc((size_t)n_s*Z, sizeof(double));
  o->dE = (double *)calloc((size_t)n_s*Z, sizeof(double));
  o->dP = (double *)calloc((size_t)n_s*Z*3, sizeof(double));
  o->N_out = (double *)calloc(n_s, sizeof(double));
  o->E_out = (double *)calloc(n_s, sizeof(double));
  return o;
}

void orc_destroy(orc_t *o) {
  if (!o) return;
  free(o->r_e); free(o->th_e); free(o->kind); free(o->e_e); free(o->e_c); free(o->dGam);
  free(o->mu); free(o->dmu); free(o->Phc); free(o->dOm); free(o->vol); free(o->f);
  free(o->v); free(o->v0); free(o->al); free(o->al0); free(o->ph); free(o->ph0);
  free(o->ka); free(o->ks); free(o->fe); free(o->dN); free(o->dE); free(o->dP);
  free(o->N_out); free(o->E_out); free(o->fbc); free(o);
}

/* [R-18] a background set after another one marks a time remap for the next
 * step (from the previous background's frames to the new one's). */
void orc_set_background(orc_t *o, const double *v, const double *al, const double *ph,
                        const double *ka, const double *ks, const double *fe) {
  int Z = nz(o);
  if (o->has_bg) {
    memcpy(o->v0, o->v, sizeof(double)*3*Z);
    memcpy(o->al0, o->al, sizeof(double)*Z);
    memcpy(o->ph0, o->ph, sizeof(double)*Z);
    o->remap_pending = 1;
    o->has_prev = 1;
  }
  memcpy(o->v, v, sizeof(double)*3*Z);
  memcpy(o->al, al, sizeof(double)*Z);
  memcpy(o->ph, ph, sizeof(double)*Z);
  size_t NO = (size_t)o->n_s * Z * o->n_e;
  memcpy(o->ka, ka, sizeof(double)*NO);
  memcpy(o->ks, ks, sizeof(double)*NO);
  memcpy(o->fe, fe, sizeof(double)*NO);
  o->has_bg = 1;
}

/* [R-15b] distribution imposed on the incoming bins of the open face at
 * th_max (isotropic in the face's comoving frame), [s][radial zone][group] */
void orc_set_boundary(orc_t *o, const double *fbc) {
  memcpy(o->fbc, fbc, sizeof(double) * (size_t)o->n_s * o->n_r * o->n_e);
}

void orc_set_f(orc_t *o, const double *f) {
  memcpy(o->f, f, sizeof(double) * (size_t)o->n_s * nz(o) * nrow(o));
  o->remap_pending = 0;
}
void orc_get_f(const orc_t *o, double *f) {
  memcpy(f, o->f, sizeof(double) * (size_t)o->n_s * nz(o) * nrow(o));
}

/* comoving unit direction of angle bin (j,k): (mu, sqrt(1-mu^2) cos Phi,
 * sqrt(1-mu^2) sin Phi) in the local (r, theta, phi) triad (Sec. 3.1) */
static void bin_dir(const orc_t *o, int ang, double *n) {
  int j = ang / o->n_ph, k = ang % o->n_ph;
  double s = sqrt(1.0 - o->mu[j]*o->mu[j]);
  n[0] = o->mu[j]; n[1] = s*cos(o->Phc[k]); n[2] = s*sin(o->Phc[k]);
}

/* Eulerian energy factor u^0 of the comoving unit vector: gamma (1 + v.n) */
static double u0_of(const double *v, const double *n) {
  double g = 1.0 / sqrt(1.0 - dot3(v, v));
  return g * (1.0 + dot3(v, n));
}

/* A location with a frame: triad angles, fluid velocity (own triad), lapse,
 * conformal factor.  Cells, faces and periodic images are all locations. */
typedef struct { double th, ph; double v[3]; double al, cf; } loc_t;

/* Remap operator T_{X->Y} (Sec. 3.2): for each source bin (i, j, k) the
 * content src[i][ang] is deposited, times `scale`, into the eight destination
 * bins bracketing (eps*, mu*, Phi*) with trilinear weights; dst += T[src].
 * [R-5] T acts on content (number), so number is conserved exactly. */
static void remap(orc_t *o, const loc_t *X, const loc_t *Y, int axis,
                  const double *src, double *dst, double scale) {
  double G[9];
  long n_tir = 0, n_ce = 0, n_cm = 0;   /* diagnostics of this call */
  orc_rotation(X->th, X->ph, Y->th, Y->ph, G);
  for (int ang = 0; ang < o->n_ang; ++ang) {
    double n[3], rho, mus, Phis;
    bin_dir(o, ang, n);
    n_tir += orc_chain(X->v, X->al, X->cf, Y->v, Y->al, Y->cf, G, axis, n, &rho, &mus, &Phis);
    int m, jL, kL;
    double we, wm, wp;
    orc_weights_eps(rho, o->R, &m, &we);
    orc_weights_mu(mus, o->n_mu, o->mu, &jL, &wm);
    orc_weights_phi(Phis, o->n_ph, &kL, &wp);
    if (o->n_mu > 1 && (mus < o->mu[0] || mus > o->mu[o->n_mu-1])) n_cm++;
    int jR = o->n_mu > 1 ? jL + 1 : jL;
    int kR = (kL + 1) % o->n_ph;
    for (int i = 0; i < o->n_e; ++i) {
      double c = scale * src[(size_t)i*o->n_ang + ang];
      if (c == 0.0) continue;
      for (int ie = 0; ie < 2; ++ie) {
        int it = i + m + ie;
        double w1 = ie ? we : 1.0 - we;
        if ((it < 0 || it > o->n_e - 1) && w1 != 0.0) n_ce++;
        if (it < 0) it = 0;
        if (it > o->n_e - 1) it = o->n_e - 1;
        for (int ij = 0; ij < 2; ++ij) {
          int jt = ij ? jR : jL;
          double w2 = ij ? wm : 1.0 - wm;
          if (o->lobatto && (jt == 0 || jt == o->n_mu - 1)) {
            /* [R-2b] a pole node (mu = +-1): its N_Phi cells are one
             * direction, so the content is spread evenly over them */
            for (int kt = 0; kt < o->n_ph; ++kt)
              dst[(size_t)it*o->n_ang + jt*o->n_ph + kt] += w1*w2*c / o->n_ph;
            continue;
          }
          for (int ik = 0; ik < 2; ++ik) {
            int kt = ik ? kR : kL;
            double w3 = ik ? wp : 1.0 - wp;
            dst[(size_t)it*o->n_ang + jt*o->n_ph + kt] += w1*w2*w3*c;
          }
        }
      }
    }
  }
#ifdef _OPENMP
#pragma omp atomic
#endif
  o->n_tir += (int)n_tir;
#ifdef _OPENMP
#pragma omp atomic
#endif
  o->n_clamp_e += n_ce;
#ifdef _OPENMP
#pragma omp atomic
#endif
  o->n_clamp_mu += n_cm;
}

/* density of bin content per coordinate volume: phi^6 u^0 dGamma dOmega f
 * (Sec. 3.1, number N in the CFC metric) */
static void to_density(const orc_t *o, const loc_t *X, const double *f, double *d) {
  double c6 = pow(X->cf, 6);
  for (int ang = 0; ang < o->n_ang; ++ang) {
    double n[3];
    bin_dir(o, ang, n);
    double u0 = u0_of(X->v, n);
    for (int i = 0; i < o->n_e; ++i)
      d[(size_t)i*o->n_ang + ang] = c6 * u0 * o->dGam[i] * o->dOm[ang] * f[(size_t)i*o->n_ang + ang];
  }
}
static void from_density(const orc_t *o, const loc_t *X, const double *d, double *f) {
  double c6 = pow(X->cf, 6);
  for (int ang = 0; ang < o->n_ang; ++ang) {
    double n[3];
    bin_dir(o, ang, n);
    double u0 = u0_of(X->v, n);
    for (int i = 0; i < o->n_e; ++i)
      f[(size_t)i*o->n_ang + ang] = d[(size_t)i*o->n_ang + ang] / (c6 * u0 * o->dGam[i] * o->dOm[ang]);
  }
}

/* ------------------------------------------------------------------------- */
/* Face description                                                          */
/* ------------------------------------------------------------------------- */
enum { FACE_INTERNAL = 0, FACE_OUTFLOW_P = 1, FACE_OUTFLOW_Q = 2, FACE_REFLECT_Q = 3 };

typedef struct {
  int type, axis;          /* axis: 0 r (or z), 1 theta, 2 phi */
  int z[4];                /* zones of P-1, P, Q, Q+1 (-1: absent) */
  loc_t L[4];              /* their frames/backgrounds at this face */
  double x[4];             /* 1D positions along the stencil */
  loc_t S;                 /* face frame and background */
  double xs, area;
  int imposed;             /* open face whose incoming bins take fbc of radial zone `ra` */
  int ra;
} face_t;

static void zone_loc(const orc_t *o, int zone, double th, double ph, loc_t *L) {
  L->th = th; L->ph = ph;
  for (int i = 0; i < 3; ++i) L->v[i] = o->v[3*zone + i];
  L->al = o->al[zone]; L->cf = o->ph[zone];
}

static double th_c(const orc_t *o, int b) { return 0.5*(o->th_e[b] + o->th_e[b+1]); }
static double r_c(const orc_t *o, int a) { return 0.5*(o->r_e[a] + o->r_e[a+1]); }

/* Face frame and background.  [R-8b] the face triad is taken at the
 * direction whose triad axis along the stepping coordinate is the exact
 * normal of the flat face; [R-12] alpha, phi and v at the face are the means
 * of the two neighbours (v rotated into the face triad first); for boundary
 * faces the present cell's values (normal velocity set to 0 at a reflecting
 * wall). */
static void face_background(face_t *F) {
  int P = F->z[1], Q = F->z[2];
  double G[9], vp[3] = {0, 0, 0}, vq[3] = {0, 0, 0};
  if (P >= 0) {
    orc_rotation(F->L[1].th, F->L[1].ph, F->S.th, F->S.ph, G);
    for (int m = 0; m < 3; ++m) vp[m] = G[3*m]*F->L[1].v[0] + G[3*m+1]*F->L[1].v[1] + G[3*m+2]*F->L[1].v[2];
  }
  if (Q >= 0) {
    orc_rotation(F->L[2].th, F->L[2].ph, F->S.th, F->S.ph, G);
    for (int m = 0; m < 3; ++m) vq[m] = G[3*m]*F->L[2].v[0] + G[3*m+1]*F->L[2].v[1] + G[3*m+2]*F->L[2].v[2];
  }
  if (P >= 0 && Q >= 0) {
    for (int m = 0; m < 3; ++m) F->S.v[m] = 0.5*(vp[m] + vq[m]);
    F->S.al = 0.5*(F->L[1].al + F->L[2].al);
    F->S.cf = 0.5*(F->L[1].cf + F->L[2].cf);
  } else if (P >= 0) {
    for (int m = 0; m < 3; ++m) F->S.v[m] = vp[m];
    F->S.al = F->L[1].al; F->S.cf = F->L[1].cf;
  } else {
    for (int m = 0; m < 3; ++m) F->S.v[m] = vq[m];
    F->S.al = F->L[2].al; F->S.cf = F->L[2].cf;
    if (F->type == FACE_REFLECT_Q) F->S.v[F->axis] = 0.0;
  }
}

/* Radial face at edge a of row b (between zones a-1 and a). */
static int make_r_face(orc_t *o, int b, int a, face_t *F) {
  memset(F, 0, sizeof(*F));
  F->axis = 0;
  double thc = th_c(o, b);
  double dph = o->dphi;
  int slab = o->geom == ORC_SLAB;
  F->area = slab ? 1.0 : orc_face_area_r(o->r_e[a], o->th_e[b], o->th_e[b+1], dph);
  if (F->area == 0.0) return 0;
  if (a == 0) F->type = slab ? FACE_OUTFLOW_Q : FACE_REFLECT_Q;
  else if (a == o->n_r) F->type = FACE_OUTFLOW_P;
  else F->type = FACE_INTERNAL;
  for (int s = 0; s < 4; ++s) {
    int aa = a - 2 + s;
    F->z[s] = (aa >= 0 && aa < o->n_r) ? b*o->n_r + aa : -1;
    if (F->z[s] >= 0) {
      zone_loc(o, F->z[s], slab ? 0.0 : thc, 0.0, &F->L[s]);
      F->x[s] = r_c(o, aa);
    }
  }
  /* r-face triad: colatitude of the flat face's normal */
  F->S.th = slab ? 0.0 : atan2(sin(thc), cos(thc)*cos(0.5*dph));
  F->S.ph = 0.0;
  F->xs = o->r_e[a];
  face_background(F);
  return 1;
}

/* Polar face of a 2D grid at edge bf (between rows bf-1 and bf), radius a.
 * bf == n_th with th_max < pi: the open face at th_max (P = the last row);
 * outgoing bins leave, incoming bins take the imposed fbc [R-15b]. */
static int make_th_face(orc_t *o, int a, int bf, face_t *F) {
  memset(F, 0, sizeof(*F));
  F->axis = 1;
  F->type = FACE_INTERNAL;
  if (bf == o->n_th) {
    F->type = FACE_OUTFLOW_P;
    F->imposed = 1;
    F->ra = a;
  }
  double the = o->th_e[bf], rc = r_c(o, a);
  F->area = orc_face_area_th(o->r_e[a], o->r_e[a+1], the, o->dphi);
  if (F->area == 0.0) return 0;
  for (int s = 0; s < 4; ++s) {
    int bb = bf - 2 + s;
    F->z[s] = (bb >= 0 && bb < o->n_th) ? bb*o->n_r + a : -1;
    if (F->z[s] >= 0) {
      zone_loc(o, F->z[s], th_c(o, bb), 0.0, &F->L[s]);
      F->x[s] = rc * th_c(o, bb);
    }
  }
  F->S.th = atan2(sin(the)*cos(0.5*o->dphi), cos(the));
  F->S.ph = 0.0;
  F->xs = rc * the;
  face_background(F);
  return 1;
}

/* Periodic lateral face of zone z in a column (axis 1) or wedge (axis 2):
 * the stencil is the zone itself seen at offsets -1, 0, +1, +2 steps. */
static int make_periodic_face(orc_t *o, int zone, int axis, face_t *F) {
  memset(F, 0, sizeof(*F));
  F->axis = axis;
  F->type = FACE_INTERNAL;
  int a = zone % o->n_r, b = zone / o->n_r;
  double thc = th_c(o, b), rc = r_c(o, a);
  if (axis == 1) {
    double d = o->dth_col;
    double the = thc + 0.5*d;
    F->area = orc_face_area_th(o->r_e[a], o->r_e[a+1], the, o->dphi);
    for (int s = 0; s < 4; ++s) {
      F->z[s] = zone;
      zone_loc(o, zone, thc + (s - 1)*d, 0.0, &F->L[s]);
      F->x[s] = rc * (thc + (s - 1)*d);
    }
    F->S.th = atan2(sin(the)*cos(0.5*o->dphi), cos(the));
    F->S.ph = 0.0;
    F->xs = rc * the;
  } else {
    double d = o->dphi;
    F->area = orc_face_area_ph(o->r_e[a], o->r_e[a+1], o->th_e[b], o->th_e[b+1], 0.5*d);
    double rs = rc * sin(thc);
    for (int s = 0; s < 4; ++s) {
      F->z[s] = zone;
      zone_loc(o, zone, thc, (s - 1)*d, &F->L[s]);
      F->x[s] = rs * (s - 1)*d;
    }
    F->S.th = thc;
    F->S.ph = 0.5*d;
    F->xs = rs * 0.5*d;
  }
  if (F->area == 0.0) return 0;
  face_background(F);
  return 1;
}

/* ------------------------------------------------------------------------- */
/* Interface distribution and flux for one species (Sec. 3.3)                */
/* Flux[i][ang] = content crossing the face from P to Q during dt, per face  */
/* bin: dt dA phi^6 (alpha/phi^2) u^n dGamma dOmega f_s   (Sec. 3.1, F).     */
/* ------------------------------------------------------------------------- */
static void face_flux(orc_t *o, const face_t *F, int s, double dt, double *flux) {
  size_t R = nrow(o);
  int Z = nz(o);
  double *d = (double *)malloc(sizeof(double) * R);
  double *D = (double *)malloc(sizeof(double) * R);
  double *g[4];
  for (int k = 0; k < 4; ++k) g[k] = (double *)calloc(R, sizeof(double));
  int present[4];
  for (int k = 0; k < 4; ++k) {
    present[k] = F->z[k] >= 0;
    if (!present[k]) continue;
    /* remap the stencil cell's content into the face frame, then express
     * it as the distribution function at the face: g = T_{X->s}[n_X] */
    to_density(o, &F->L[k], o->f + ((size_t)s*Z + F->z[k])*R, d);
    memset(D, 0, sizeof(double) * R);
    remap(o, &F->L[k], &F->S, F->axis, d, D, 1.0);
    from_density(o, &F->S, D, g[k]);
  }
  /* face bins: Eulerian energy factor and normal coordinate velocity
   * v_b = alpha phi^-2 u^n / u^0 */
  double *u0 = (double *)malloc(sizeof(double) * o->n_ang);
  double *vn = (double *)malloc(sizeof(double) * o->n_ang);
  for (int ang = 0; ang < o->n_ang; ++ang) {
    double n[3], u[4] = {1, 0, 0, 0}, ue[4];
    bin_dir(o, ang, n);
    u[1] = n[0]; u[2] = n[1]; u[3] = n[2];
    orc_boost(F->S.v, +1, u, ue);
    u0[ang] = ue[0];
    vn[ang] = F->S.al / (F->S.cf*F->S.cf) * ue[1+F->axis] / ue[0];
  }
  double *fs = (double *)calloc(R, sizeof(double));
  if (F->type == FACE_INTERNAL) {
    double dx = F->x[2] - F->x[1];
    double *r = (double *)malloc(sizeof(double) * o->n_ang);
    double *tau = (double *)malloc(sizeof(double) * o->n_ang);
    double *flw = (double *)malloc(sizeof(double) * o->n_ang);
    for (int i = 0; i < o->n_e; ++i) {
      size_t zP = (size_t)s*Z + F->z[1], zQ = (size_t)s*Z + F->z[2];
      double ka = 0.5*(o->ka[zP*o->n_e + i] + o->ka[zQ*o->n_e + i]);
      double ks = 0.5*(o->ks[zP*o->n_e + i] + o->ks[zQ*o->n_e + i]);
      double fe = 0.5*(o->fe[zP*o->n_e + i] + o->fe[zQ*o->n_e + i]);
      /* Lax-Wendroff half step (Eq. halfstep) with the collision term
       * implicit at n+1/2 [R-10], lab-time factor alpha/u^0 [R-17] */
      for (int ang = 0; ang < o->n_ang; ++ang) {
        size_t q = (size_t)i*o->n_ang + ang;
        tau[ang] = 0.5*dt * F->S.al / u0[ang];
        r[ang] = 0.5*(g[1][q] + g[2][q]) - 0.5*dt*vn[ang]*(g[2][q] - g[1][q])/dx
                 + tau[ang]*ka*fe;
      }
      orc_collision_row(o->n_ang, r, tau, ka, ks, o->dOm, flw);
      /* flux-switch weight (Sec. 3.3.3), per group: exp(-(ka+ks) dx) with the
       * opacity of the cell the particles arrive from (the upwind cell) [R-12b] */
      double kP = o->ka[zP*o->n_e + i] + o->ks[zP*o->n_e + i];
      double kQ = o->ka[zQ*o->n_e + i] + o->ks[zQ*o->n_e + i];
      double wP = exp(-kP*dx), wQ = exp(-kQ*dx);
      for (int ang = 0; ang < o->n_ang; ++ang) {
        size_t q = (size_t)i*o->n_ang + ang;
        /* upwind with MC-limited linear reconstruction (Sec. 3.3.2) [R-11] */
        double fu;
        if (vn[ang] >= 0.0) {
          double sl = 0.0;
          if (present[0]) sl = mc_limiter((g[1][q] - g[0][q])/(F->x[1] - F->x[0]),
                                          (g[2][q] - g[1][q])/(F->x[2] - F->x[1]));
          fu = g[1][q] + sl*(F->xs - F->x[1]);
        } else {
          double sl = 0.0;
          if (present[3]) sl = mc_limiter((g[2][q] - g[1][q])/(F->x[2] - F->x[1]),
                                          (g[3][q] - g[2][q])/(F->x[3] - F->x[2]));
          fu = g[2][q] + sl*(F->xs - F->x[2]);
        }
        double w = vn[ang] >= 0.0 ? wP : wQ;
        fs[q] = (1.0 - w)*flw[ang] + w*fu;
      }
    }
    free(r); free(tau); free(flw);
  } else if (F->type == FACE_OUTFLOW_P || F->type == FACE_OUTFLOW_Q) {
    /* [R-15] open boundary: outgoing bins take the present cell's value,
     * incoming bins see vacuum */
    int k = F->type == FACE_OUTFLOW_P ? 1 : 2;
    for (int i = 0; i < o->n_e; ++i) {
      double fin = F->imposed ? o->fbc[((size_t)s*o->n_r + F->ra)*o->n_e + i] : 0.0;
      for (int ang = 0; ang < o->n_ang; ++ang) {
        size_t q = (size_t)i*o->n_ang + ang;
        int out = F->type == FACE_OUTFLOW_P ? (vn[ang] >= 0.0) : (vn[ang] < 0.0);
        fs[q] = out ? g[k][q] : fin;
      }
    }
  } else { /* FACE_REFLECT_Q: specular wall at rest [R-15] */
    for (int i = 0; i < o->n_e; ++i)
      for (int ang = 0; ang < o->n_ang; ++ang) {
        int j = ang / o->n_ph, kk = ang % o->n_ph;
        size_t q = (size_t)i*o->n_ang + ang;
        size_t qm = (size_t)i*o->n_ang + (o->n_mu - 1 - j)*o->n_ph + kk;
        fs[q] = vn[ang] < 0.0 ? g[2][q] : g[2][qm];
      }
  }
  double c6 = pow(F->S.cf, 6);
  for (int i = 0; i < o->n_e; ++i)
    for (int ang = 0; ang < o->n_ang; ++ang) {
      size_t q = (size_t)i*o->n_ang + ang;
      flux[q] = dt * F->area * c6 * u0[ang] * vn[ang] * o->dGam[i] * o->dOm[ang] * fs[q];
    }
  free(fs); free(u0); free(vn); free(d); free(D);
  for (int k = 0; k < 4; ++k) free(g[k]);
}

/* Deposits of one face's flux into its two neighbours' content changes
 * (Eq. fullstep): depP = -T_{s->P}[F], depQ = +T_{s->Q}[F], into zeroed
 * buffers of their own; tally[0..1] = the number and the energy at infinity
 * (alpha eps u^0 per unit number) that left through an open boundary.
 * [R-13] */
static void face_deposit(orc_t *o, const face_t *F, const double *flux, double *depP, double *depQ,
                         double *tally) {
  size_t R = nrow(o);
  memset(depP, 0, sizeof(double) * R);
  memset(depQ, 0, sizeof(double) * R);
  if (F->z[1] >= 0) remap(o, &F->S, &F->L[1], F->axis, flux, depP, -1.0);
  if (F->z[2] >= 0) remap(o, &F->S, &F->L[2], F->axis, flux, depQ, +1.0);
  tally[0] = tally[1] = 0.0;
  if (F->type == FACE_OUTFLOW_P || F->type == FACE_OUTFLOW_Q) {
    double sg = F->type == FACE_OUTFLOW_P ? 1.0 : -1.0;
    for (int ang = 0; ang < o->n_ang; ++ang) {
      double n[3];
      bin_dir(o, ang, n);
      double u0 = u0_of(F->S.v, n);
      for (int i = 0; i < o->n_e; ++i) {
        double c = sg * flux[(size_t)i*o->n_ang + ang];
        tally[0] += c;
        tally[1] += c * F->S.al * o->e_c[i] * u0;
      }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Time remap T_{n->n+1} (Sec. 3.2): per zone, old frame -> new frame, G = I. */
/* ------------------------------------------------------------------------- */
static void time_remap(orc_t *o) {
  int Z = nz(o);
  size_t R = nrow(o);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    double *d = (double *)malloc(sizeof(double) * R);
    double *D = (double *)malloc(sizeof(double) * R);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int z = 0; z < Z; ++z) {
      loc_t X, Y;
      X.th = Y.th = 0.0; X.ph = Y.ph = 0.0;
      for (int m = 0; m < 3; ++m) { X.v[m] = o->v0[3*z+m]; Y.v[m] = o->v[3*z+m]; }
      X.al = o->al0[z]; X.cf = o->ph0[z];
      Y.al = o->al[z]; Y.cf = o->ph[z];
      for (int s = 0; s < o->n_s; ++s) {
        double *f = o->f + ((size_t)s*Z + z)*R;
        to_density(o, &X, f, d);
        memset(D, 0, sizeof(double) * R);
        remap(o, &X, &Y, KICK_TIME, d, D, 1.0);
        from_density(o, &Y, D, f);
      }
    }
    free(d); free(D);
  }
}

/* enumerate every face once: returns the number written to `faces` */
static int build_faces(orc_t *o, face_t **out) {
  int cap = 8 + 4 * nz(o) + 2 * o->n_th * (o->n_r + 1) + 2 * o->n_r * (o->n_th + 1);
  face_t *fc = (face_t *)malloc(sizeof(face_t) * cap);
  int n = 0;
  for (int b = 0; b < o->n_th; ++b)
    for (int a = 0; a <= o->n_r; ++a) n += make_r_face(o, b, a, &fc[n]);
  if (o->geom == ORC_SPHERICAL) {
    if (o->periodic_th) {
      for (int z = 0; z < nz(o); ++z) n += make_periodic_face(o, z, 1, &fc[n]);
    } else {
      int last = o->th_max < PI_ ? o->n_th : o->n_th - 1;   /* the open face at th_max */
      for (int a = 0; a < o->n_r; ++a)
        for (int bf = 1; bf <= last; ++bf) n += make_th_face(o, a, bf, &fc[n]);
    }
    for (int z = 0; z < nz(o); ++z) n += make_periodic_face(o, z, 2, &fc[n]);
  }
  *out = fc;
  return n;
}

/* ------------------------------------------------------------------------- */
/* One transport step (Sec. 3.3 Eq. fullstep + Sec. 3.5):                    */
/*  1. time remap if the background changed                                  */
/*  2. interface fluxes of every face from f^n, deposited unsplit           */
/*  3. f* = f^n + dN / (phi^6 dV u^0 dGamma dOmega)                         */
/*  4. implicit collision per (zone, group) -> f^{n+1}; collision moments    */
/* ------------------------------------------------------------------------- */
enum { FACE_BLOCK = 256 };   /* faces whose deposits are computed together */

/* Fluxes of the faces q with dtf[q] > 0 (each over its own dtf[q]) from the
 * current f, deposited into both neighbours' content changes dN (Eq.
 * fullstep), outflow added to the tallies. */
static void deposit_faces(orc_t *o, const face_t *faces, int nf, const double *dtf, double *dN) {
  int Z = nz(o);
  size_t R = nrow(o);
  double *flux = (double *)malloc(sizeof(double) * R * FACE_BLOCK);
  double *depP = (double *)malloc(sizeof(double) * R * FACE_BLOCK);
  double *depQ = (double *)malloc(sizeof(double) * R * FACE_BLOCK);
  double tally[2 * FACE_BLOCK];
  for (int s = 0; s < o->n_s; ++s)
    for (int q0 = 0; q0 < nf; q0 += FACE_BLOCK) {
      int nb = nf - q0 < FACE_BLOCK ? nf - q0 : FACE_BLOCK;
      /* the block's fluxes and deposits, each face on its own buffers */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
      for (int k = 0; k < nb; ++k) {
        const face_t *F = &faces[q0 + k];
        if (!(dtf[q0 + k] > 0.0)) continue;
        face_flux(o, F, s, dtf[q0 + k], flux + (size_t)k * R);
        face_deposit(o, F, flux + (size_t)k * R, depP + (size_t)k * R, depQ + (size_t)k * R, tally + 2 * k);
      }
      /* added to the zones in face-list order */
      for (int k = 0; k < nb; ++k) {
        if (!(dtf[q0 + k] > 0.0)) continue;
        const face_t *F = &faces[q0 + k];
        for (int side = 1; side <= 2; ++side) {
          if (F->z[side] < 0) continue;
          double *d = dN + ((size_t)s*Z + F->z[side])*R;
          const double *src = (side == 1 ? depP : depQ) + (size_t)k * R;
          for (size_t q = 0; q < R; ++q) d[q] += src[q];
        }
        if (F->type == FACE_OUTFLOW_P || F->type == FACE_OUTFLOW_Q) {
          o->N_out[s] += tally[2 * k];
          o->E_out[s] += tally[2 * k + 1];
        }
      }
    }
  free(flux); free(depP); free(depQ);
}

/* Collision of the zones with dtz[z] > 0 (Sec. 3.5) over their own dtz[z]:
 * f* = f + dN / (phi^6 dV u^0 dGamma dOmega), the implicit solve, f^{n+1}
 * into dst (o->f, or `out` in subset mode); the zone's dN rows are then
 * spent (zeroed).  Moments (Eq. hydrosource): the content change over dtz
 * per unit volume, per unit of `tm` (the time the moments average over):
 * written (acc = 0) or added (acc = 1). */
static void collide_zones(orc_t *o, const double *dtz, double *dN, double *out, double tm, int acc) {
  int Z = nz(o);
  size_t R = nrow(o);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    double *r = (double *)malloc(sizeof(double) * o->n_ang);
    double *tau = (double *)malloc(sizeof(double) * o->n_ang);
    double *fst = (double *)malloc(sizeof(double) * o->n_ang);
    double *fnew = (double *)malloc(sizeof(double) * o->n_ang);
    double *u0 = (double *)malloc(sizeof(double) * o->n_ang);
    double *nd = (double *)malloc(sizeof(double) * 3 * o->n_ang);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
    for (int z = 0; z < Z; ++z) {
      double dt = dtz[z];
      if (!(dt > 0.0)) continue;
      loc_t X;
      zone_loc(o, z, 0.0, 0.0, &X);
      for (int ang = 0; ang < o->n_ang; ++ang) {
        bin_dir(o, ang, nd + 3*ang);
        u0[ang] = u0_of(X.v, nd + 3*ang);
        tau[ang] = X.al * dt / u0[ang];       /* [R-17] */
      }
      double c6 = pow(X.cf, 6);
      for (int s = 0; s < o->n_s; ++s) {
        double sN = 0.0, sE = 0.0, sP[3] = {0, 0, 0};
        for (int i = 0; i < o->n_e; ++i) {
          size_t zo = ((size_t)s*Z + z)*o->n_e + i;
          double ka = o->ka[zo], ks = o->ks[zo], fe = o->fe[zo];
          size_t base = ((size_t)s*Z + z)*R + (size_t)i*o->n_ang;
          const double *f = o->f + base;
          double *dn = dN + base;
          for (int ang = 0; ang < o->n_ang; ++ang) {
            fst[ang] = f[ang] + dn[ang] / (c6 * o->vol[z] * u0[ang] * o->dGam[i] * o->dOm[ang]);
            r[ang] = fst[ang] + tau[ang]*ka*fe;
            dn[ang] = 0.0;
          }
          orc_collision_row(o->n_ang, r, tau, ka, ks, o->dOm, fnew);
          double *dst = out ? out + base : o->f + base;
          for (int ang = 0; ang < o->n_ang; ++ang) {
            /* collision moments (Eq. hydrosource) [R-17]: content change per
             * coordinate volume and time */
            double dc = c6 * u0[ang] * o->dGam[i] * o->dOm[ang] * (fnew[ang] - fst[ang]) / tm;
            sN += dc;
            sE += dc * o->e_c[i];
            for (int m = 0; m < 3; ++m) sP[m] += dc * o->e_c[i] * nd[3*ang+m];
            dst[ang] = fnew[ang];
          }
        }
        size_t q = (size_t)s*Z + z;
        if (acc) {
          o->dN[q] += sN; o->dE[q] += sE;
          for (int m = 0; m < 3; ++m) o->dP[q*3 + m] += sP[m];
        } else {
          o->dN[q] = sN; o->dE[q] = sE;
          for (int m = 0; m < 3; ++m) o->dP[q*3 + m] = sP[m];
        }
      }
    }
    free(r); free(tau); free(fst); free(fnew); free(u0); free(nd);
  }
}

static void step_impl(orc_t *o, double dt, const int *sel, double *out) {
  int Z = nz(o);
  size_t R = nrow(o);
  if (o->remap_pending) { time_remap(o); o->remap_pending = 0; }
  face_t *faces;
  int nf = build_faces(o, &faces);
  double *dN = (double *)calloc((size_t)o->n_s * Z * R, sizeof(double));
  double *dtf = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  double *dtz = (double *)malloc(sizeof(double) * Z);
  for (int q = 0; q < nf; ++q) {
    dtf[q] = dt;
    if (sel) {  /* subset mode: only faces that touch a selected zone */
      int zp = faces[q].z[1], zq = faces[q].z[2];
      if (!((zp >= 0 && sel[zp]) || (zq >= 0 && sel[zq]))) dtf[q] = 0.0;
    }
  }
  for (int z = 0; z < Z; ++z) dtz[z] = (sel && !sel[z]) ? 0.0 : dt;
  deposit_faces(o, faces, nf, dtf, dN);
  collide_zones(o, dtz, dN, sel ? out : NULL, dt, 0);
  free(dN); free(faces); free(dtf); free(dtz);
}

/* ------------------------------------------------------------------------- */
/* Local time stepping (Sec. 5: "the timestep can be much larger in the      */
/* larger outer zones") [R-19]: zone z advances with dt0 2^lev[z], lev in     */
/* [0, L); one call advances every zone by the macro step dt0 2^(L-1).  At   */
/* substep k (of dt0) a face whose finer side has level l = min(lev_P,      */
/* lev_Q) is evaluated when k is a multiple of 2^l, over dt0 2^l, from the   */
/* current f (a coarser neighbour's f is still that of the start of its own */
/* step); its deposit goes to both sides, where it waits until the side's   */
/* step ends (Eq. fullstep; number conserved face by face).  A zone whose    */
/* step ends at substep k, (k + 1) a multiple of 2^lev, then takes its        */
/* collision over its own step (Sec. 3.5).  Moments are averaged over the   */
/* macro step.  The time remap runs once, before the first substep.         */
/* ------------------------------------------------------------------------- */
int orc_step_lts(orc_t *o, double dt0, const int *lev, int L) {
  int Z = nz(o);
  size_t R = nrow(o);
  if (L < 1 || L > 16) return -1;
  for (int z = 0; z < Z; ++z) if (lev[z] < 0 || lev[z] >= L) return -1;
  if (o->remap_pending) { time_remap(o); o->remap_pending = 0; }
  face_t *faces;
  int nf = build_faces(o, &faces);
  double *dN = (double *)calloc((size_t)o->n_s * Z * R, sizeof(double));
  double *dtf = (double *)malloc(sizeof(double) * (nf > 0 ? nf : 1));
  double *dtz = (double *)malloc(sizeof(double) * Z);
  const int K = 1 << (L - 1);
  const double tm = dt0 * K;
  for (size_t q = 0; q < (size_t)o->n_s * Z; ++q) o->dN[q] = o->dE[q] = 0.0;
  for (size_t q = 0; q < (size_t)o->n_s * Z * 3; ++q) o->dP[q] = 0.0;
  for (int k = 0; k < K; ++k) {
    for (int q = 0; q < nf; ++q) {
      int zp = faces[q].z[1], zq = faces[q].z[2];
      int l = zp >= 0 ? lev[zp] : lev[zq];
      if (zp >= 0 && zq >= 0 && lev[zq] < l) l = lev[zq];
      dtf[q] = (k % (1 << l)) == 0 ? dt0 * (1 << l) : 0.0;
    }
    for (int z = 0; z < Z; ++z) dtz[z] = ((k + 1) % (1 << lev[z])) == 0 ? dt0 * (1 << lev[z]) : 0.0;
    deposit_faces(o, faces, nf, dtf, dN);
    collide_zones(o, dtz, dN, NULL, tm, 1);
  }
  free(dN); free(faces); free(dtf); free(dtz);
  return 0;
}

/* [R-19] Levels of the local time stepping: dt0 = cfl / max rate; zone z
 * takes the largest l < max_levels whose step dt0 2^l stays within its own
 * limit cfl / rate[z]; then levels are lowered until zones that share a
 * radial face (or, on 2D grids, a polar face) differ by at most one level.
 * Returns dt0 and writes lev[zone]. */
void orc_zone_rates(orc_t *o, double *zr);
double orc_lts_levels(orc_t *o, double cfl, int max_levels, int *lev) {
  int Z = nz(o);
  double *zr = (double *)malloc(sizeof(double) * Z);
  orc_zone_rates(o, zr);
  double mx = 0.0;
  for (int z = 0; z < Z; ++z) if (zr[z] > mx) mx = zr[z];
  for (int z = 0; z < Z; ++z) {
    int l = 0;
    /* dt0 2^(l+1) <= cfl / rate  <=>  rate 2^(l+1) <= mx */
    while (l + 1 < max_levels && zr[z] * (double)(1 << (l + 1)) <= mx) ++l;
    lev[z] = l;
  }
  int polar = o->geom == ORC_SPHERICAL && !o->periodic_th && o->n_th > 1;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int z = 0; z < Z; ++z) {
      int a = z % o->n_r, b = z / o->n_r, l = lev[z];
      if (a > 0 && lev[z - 1] + 1 < l) l = lev[z - 1] + 1;
      if (a + 1 < o->n_r && lev[z + 1] + 1 < l) l = lev[z + 1] + 1;
      if (polar && b > 0 && lev[z - o->n_r] + 1 < l) l = lev[z - o->n_r] + 1;
      if (polar && b + 1 < o->n_th && lev[z + o->n_r] + 1 < l) l = lev[z + o->n_r] + 1;
      if (l != lev[z]) { lev[z] = l; changed = 1; }
    }
  }
  free(zr);
  return cfl / mx;
}

/* Per-zone Courant rate (the quantity orc_max_dt maximises) [R-14]: rate[z]
 * = max over bins of sum over faces of max(0, u.n_out) dA / dV. */
int orc_step(orc_t *o, double dt) {
  step_impl(o, dt, NULL, NULL);
  return 0;
}

/* Subset step for sampled checks at large sizes: computes f^{n+1} of the
 * zones flagged in sel[zone] into out (same layout as f; other zones left
 * untouched) without advancing the stored state, apart from a pending time
 * remap, which is applied to every zone. */
int orc_step_zones(orc_t *o, double dt, const int *sel, double *out) {
  step_impl(o, dt, sel, out);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------- */
/* [R-14] Courant limit: no bin of any zone may lose more than CFL of its
 * content in one step: dt <= CFL / max_{zone,bin} sum_faces max(0, u.n_out)
 * dA / dV, with u the coordinate velocity of the zone's bin expressed in the
 * face triad.  Zero-area faces do not count. */
void orc_zone_rates(orc_t *o, double *zr) {
  face_t *faces;
  int nf = build_faces(o, &faces);
  int Z = nz(o);
  double *rate = (double *)calloc((size_t)Z * o->n_ang, sizeof(double));
  for (int q = 0; q < nf; ++q) {
    face_t *F = &faces[q];
    for (int side = 1; side <= 2; ++side) {
      int z = F->z[side];
      if (z < 0) continue;
      double sg = side == 1 ? 1.0 : -1.0;   /* outward normal sign */
      double G[9];
      orc_rotation(F->L[side].th, F->L[side].ph, F->S.th, F->S.ph, G);
      for (int ang = 0; ang < o->n_ang; ++ang) {
        double n[3], u[4] = {1, 0, 0, 0}, ue[4], pn;
        bin_dir(o, ang, n);
        u[1] = n[0]; u[2] = n[1]; u[3] = n[2];
        orc_boost(F->L[side].v, +1, u, ue);
        pn = G[3*F->axis]*ue[1] + G[3*F->axis+1]*ue[2] + G[3*F->axis+2]*ue[3];
        double vel = sg * F->L[side].al / (F->L[side].cf*F->L[side].cf) * pn / ue[0];
        if (vel > 0.0) rate[(size_t)z*o->n_ang + ang] += vel * F->area / o->vol[z];
      }
    }
  }
  for (int z = 0; z < Z; ++z) {
    double mx = 0.0;
    for (int ang = 0; ang < o->n_ang; ++ang) if (rate[(size_t)z*o->n_ang + ang] > mx) mx = rate[(size_t)z*o->n_ang + ang];
    zr[z] = mx;
  }
  free(rate); free(faces);
}

/* [R-14] Courant limit: no bin of any zone may lose more than CFL of its
 * content in one step: dt <= CFL / max_{zone,bin} sum_faces max(0, u.n_out)
 * dA / dV, with u the coordinate velocity of the zone's bin expressed in the
 * face triad.  Zero-area faces do not count. */
double orc_max_dt(orc_t *o, double cfl) {
  int Z = nz(o);
  double *zr = (double *)malloc(sizeof(double) * Z);
  orc_zone_rates(o, zr);
  double mx = 0.0;
  for (int z = 0; z < Z; ++z) if (zr[z] > mx) mx = zr[z];
  free(zr);
  return cfl / mx;
}

/* Collision moments of the last step: dN, dE [s][zone], dP [s][zone][3];
 * Q_Ye [zone] = -(dN_nue - dN_nuebar) * phase_norm (Eq. hydrosource). */
void orc_moments(const orc_t *o, double *dN, double *dE, double *dP, double *QYe) {
  int Z = nz(o);
  memcpy(dN, o->dN, sizeof(double) * o->n_s * Z);
  memcpy(dE, o->dE, sizeof(double) * o->n_s * Z);
  memcpy(dP, o->dP, sizeof(double) * o->n_s * Z * 3);
  for (int z = 0; z < Z; ++z) {
    double q = 0.0;
    for (int s = 0; s < o->n_s; ++s) {
      if (o->kind[s] == 0) q -= o->dN[(size_t)s*Z + z];
      if (o->kind[s] == 1) q += o->dN[(size_t)s*Z + z];
    }
    QYe[z] = q * o->phase_norm;
  }
}

/* Totals per species: number N = sum dV phi^6 u^0 dGamma dOmega f, energy at
 * infinity E = sum dV alpha phi^6 u^0 dGamma dOmega f eps_i u^0 (the lab
 * energy of a bin is eps_i u^0), and cumulative outflow. */
void orc_totals(const orc_t *o, double *N, double *E, double *Nout, double *Eout) {
  int Z = nz(o);
  for (int s = 0; s < o->n_s; ++s) {
    double sn = 0.0, se = 0.0;
    for (int z = 0; z < Z; ++z) {
      double c6 = pow(o->ph[z], 6);
      const double *v = o->v + 3*z;
      for (int i = 0; i < o->n_e; ++i)
        for (int ang = 0; ang < o->n_ang; ++ang) {
          double n[3];
          bin_dir(o, ang, n);
          double u0 = u0_of(v, n);
          double c = o->vol[z] * c6 * u0 * o->dGam[i] * o->dOm[ang]
                     * o->f[((size_t)s*Z + z)*nrow(o) + (size_t)i*o->n_ang + ang];
          sn += c;
          se += c * o->al[z] * o->e_c[i] * u0;
        }
    }
    N[s] = sn; E[s] = se; Nout[s] = o->N_out[s]; Eout[s] = o->E_out[s];
  }
}

/* Comoving angular moments per (species, zone, group) (Sec. 4.1):
 * J = 1/4pi sum dOm f eps dGamma, H with mu, K with mu^2. */
void orc_jhk(const orc_t *o, double *J, double *H, double *K) {
  int Z = nz(o);
  for (int s = 0; s < o->n_s; ++s)
    for (int z = 0; z < Z; ++z)
      for (int i = 0; i < o->n_e; ++i) {
        double sj = 0.0, sh = 0.0, sk = 0.0;
        for (int ang = 0; ang < o->n_ang; ++ang) {
          double mu = o->mu[ang / o->n_ph];
          double c = o->dOm[ang] * o->f[((size_t)s*Z + z)*nrow(o) + (size_t)i*o->n_ang + ang]
                     * o->e_c[i] * o->dGam[i] / (4.0*PI_);
          sj += c; sh += c*mu; sk += c*mu*mu;
        }
        size_t q = ((size_t)s*Z + z)*o->n_e + i;
        J[q] = sj; H[q] = sh; K[q] = sk;
      }
}

/* accessors for tests */
void orc_grid(const orc_t *o, double *eps_c, double *dgam, double *mu, double *dmu, double *vol) {
  memcpy(eps_c, o->e_c, sizeof(double) * o->n_e);
  memcpy(dgam, o->dGam, sizeof(double) * o->n_e);
  memcpy(mu, o->mu, sizeof(double) * o->n_mu);
  memcpy(dmu, o->dmu, sizeof(double) * o->n_mu);
  memcpy(vol, o->vol, sizeof(double) * nz(o));
}
int orc_tir_count(const orc_t *o) { return o->n_tir; }

/* threads of the parallel loops (OpenMP builds; 1 otherwise) */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_clamp_counts(const orc_t *o, long *out) { out[0] = o->n_clamp_e; out[1] = o->n_clamp_mu; }

/* Flux content flux[group][angle] of face q of the step's face list (in the
 * order the step builds it: radial faces row by row, then polar, then the
 * periodic faces) for species s and step dt, from the current f; *area gets
 * the face area.  Returns 0 if q is out of range.  (Test access to the
 * interface state of Sec. 3.3.) */
int orc_face_flux(orc_t *o, int q, int s, double dt, double *flux, double *area) {
  face_t *faces;
  int nf = build_faces(o, &faces);
  int ok = q >= 0 && q < nf && s >= 0 && s < o->n_s;
  if (ok) {
    face_flux(o, &faces[q], s, dt, flux);
    *area = faces[q].area;
  }
  free(faces);
  return ok;
}

/* ------------------------------------------------------------------------- */
/* Learned-remap rows (test reference of the library's sample generator).    */
/* A row is (zone, kind, source angle).  kind 0: the zone's time remap,      */
/* previous -> current background.  kind 1 + 6 f + r: remap r of the zone's  */
/* face f (0 inner r, 1 outer r, 2 lower polar or the column's periodic      */
/* polar face, 3 upper polar, 4 azimuthal); r = 0..3 stencil cell r -> face, */
/* r = 4, 5 face -> cell 1 (P), 2 (Q).  Same faces and frames as the step    */
/* above.  Outputs the 16 features and the exact trilinear weights of        */
/* Sec. 3.2 on the offsets {-1,0,1}^3 (group, mu index, Phi index), index    */
/* 9 (de+1) + 3 (dm+1) + (dp+1), Phi offsets taken to the nearest periodic   */
/* image.  Returns 1 (usable), 2 (a nonzero weight outside the offsets;      */
/* targ = 0) or 0 (no such remap; feat = targ = 0).                          */
/* ------------------------------------------------------------------------- */
static int sur_face(orc_t *o, int zone, int fidx, face_t *F) {
  int a = zone % o->n_r, b = zone / o->n_r;
  int sph = o->geom == ORC_SPHERICAL;
  switch (fidx) {
    case 0: return make_r_face(o, b, a, F);
    case 1: return make_r_face(o, b, a + 1, F);
    case 2:
      if (!sph) return 0;
      if (o->periodic_th) return make_periodic_face(o, zone, 1, F);
      return b >= 1 ? make_th_face(o, a, b, F) : 0;
    case 3:
      if (!sph || o->periodic_th) return 0;
      return (b + 1 < o->n_th || o->th_max < PI_) ? make_th_face(o, a, b + 1, F) : 0;
    case 4:
      return sph ? make_periodic_face(o, zone, 2, F) : 0;
  }
  return 0;
}

int orc_sur_sample(orc_t *o, int zone, int kind, int ang, double *feat, double *targ) {
  for (int q = 0; q < 16; ++q) feat[q] = 0.0;
  for (int q = 0; q < 27; ++q) targ[q] = 0.0;
  if (zone < 0 || zone >= nz(o) || kind < 0 || kind > 30 || ang < 0 || ang >= o->n_ang) return 0;
  loc_t X, Y;
  int axis;
  if (kind == 0) {
    if (!o->has_prev) return 0;
    X.th = Y.th = 0.0; X.ph = Y.ph = 0.0;
    for (int m = 0; m < 3; ++m) { X.v[m] = o->v0[3*zone+m]; Y.v[m] = o->v[3*zone+m]; }
    X.al = o->al0[zone]; X.cf = o->ph0[zone];
    Y.al = o->al[zone]; Y.cf = o->ph[zone];
    axis = KICK_TIME;
  } else {
    int fidx = (kind - 1) / 6, r = (kind - 1) % 6;
    face_t F;
    if (!sur_face(o, zone, fidx, &F)) return 0;
    int slot = r < 4 ? r : r - 3;
    if (F.z[slot] < 0) return 0;
    if (r < 4) { X = F.L[slot]; Y = F.S; }
    else { X = F.S; Y = F.L[slot]; }
    axis = F.axis;
  }
  double G[9], n[3];
  orc_rotation(X.th, X.ph, Y.th, Y.ph, G);
  bin_dir(o, ang, n);
  /* features (the network's inputs) */
  for (int c = 0; c < 3; ++c) {
    feat[c] = n[c];
    feat[3+c] = X.v[c];
    feat[6+c] = G[c]*Y.v[0] + G[3+c]*Y.v[1] + G[6+c]*Y.v[2];   /* G^T v_Y */
  }
  feat[9] = 0.5*(G[7] - G[5]);
  feat[10] = 0.5*(G[2] - G[6]);
  feat[11] = 0.5*(G[3] - G[1]);
  if (axis >= 0 && axis < 3) feat[12+axis] = log(X.al / Y.al);
  feat[15] = 2.0*log(X.cf / Y.cf);
  /* exact weights */
  double rho, mus, Phis;
  orc_chain(X.v, X.al, X.cf, Y.v, Y.al, Y.cf, G, axis, n, &rho, &mus, &Phis);
  int m, jL, kL;
  double we, wm, wp;
  orc_weights_eps(rho, o->R, &m, &we);
  orc_weights_mu(mus, o->n_mu, o->mu, &jL, &wm);
  orc_weights_phi(Phis, o->n_ph, &kL, &wp);
  int j = ang / o->n_ph, k = ang % o->n_ph;
  int jR = o->n_mu > 1 ? jL + 1 : jL;
  int kR = (kL + 1) % o->n_ph;
  int rep = 1;
  for (int ie = 0; ie < 2; ++ie)
    for (int ij = 0; ij < 2; ++ij)
      for (int ik = 0; ik < 2; ++ik) {
        double c = (ie ? we : 1.0 - we) * (ij ? wm : 1.0 - wm) * (ik ? wp : 1.0 - wp);
        if (c == 0.0) continue;
        int de = m + ie, dm = (ij ? jR : jL) - j, dp = (ik ? kR : kL) - k;
        if (o->n_ph >= 3) {
          if (2*dp >= o->n_ph) dp -= o->n_ph;
          else if (2*dp < -o->n_ph) dp += o->n_ph;
        }
        if (de < -1 || de > 1 || dm < -1 || dm > 1 || dp < -1 || dp > 1) { rep = 0; continue; }
        targ[9*(de+1) + 3*(dm+1) + (dp+1)] += c;
      }
  if (!rep) {
    for (int q = 0; q < 27; ++q) targ[q] = 0.0;
    return 2;
  }
  return 1;
}

void orc_sur_samples(orc_t *o, long n, const int *idx, double *feat, double *targ, int *valid) {
  for (long i = 0; i < n; ++i)
    valid[i] = orc_sur_sample(o, idx[3*i], idx[3*i+1], idx[3*i+2], feat + 16*i, targ + 27*i);
}
