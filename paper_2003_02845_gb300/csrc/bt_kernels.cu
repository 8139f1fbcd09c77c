// bt_kernels.cu -- sm_103a kernels of the discrete-ordinate transport step
// (Chan & Mueller, arXiv:2003.02845).
//
// One CTA owns one zone (all species).  The momentum-space remap T (Sec. 3.2)
// is applied as a deterministic GATHER: for every remap the weights of each
// source angle are computed once (one thread per angle; they serve every
// group and species because the energy weights depend only on the energy
// ratio on a log-uniform group grid), source angles are bucketed by their
// lower bracket (j_L, k_L) with warp match/ballot, and every destination bin
// sums its at most four candidate buckets in a fixed order.  No atomics touch
// floating-point data, so results are bitwise reproducible.
//
// Precision: template parameter T is the arithmetic type of f, of the
// remaps and of the interface state (double for the FP64 path, float for the
// mixed path).  Content accumulators, the cell collision solve and all sums
// are float64 in both paths.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "bt_internal.h"

namespace bt {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr double kPi = 3.14159265358979323846;

// weights of one source angle for one remap
template <typename T>
struct Wt {
  T wmu, wph, we;
  short jL, kL, m, pad;
};

struct FaceDesc {
  int type, axis, own;  // own: 1 = P, 2 = Q, 3 = both (periodic face)
  int z[4];             // zone of stencil slot k (P-1, P, Q, Q+1), -1 absent
  const double* G[4];   // rotation: slot k triad -> face triad (row-major 3x3)
  double x[4], xs, dx, area;
  double v[3], al, cf;  // face background
};

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// ---------------------------------------------------------------------------
// Transformation chain (Sec. 2.2 Eq. transformchain, Sec. 3.2.2-3.2.4)
// ---------------------------------------------------------------------------
template <typename T>
struct Loc {
  T v[3];
  T g, gg;   // gamma and gamma^2/(gamma+1)
  T al, cf;
};

template <typename T>
__device__ __forceinline__ void make_loc(Loc<T>& L, const double* v, double al, double cf) {
  L.v[0] = (T)v[0]; L.v[1] = (T)v[1]; L.v[2] = (T)v[2];
  T v2 = L.v[0] * L.v[0] + L.v[1] * L.v[1] + L.v[2] * L.v[2];
  L.g = T(1) / sqrt(T(1) - v2);
  L.gg = L.g * L.g / (L.g + T(1));
  L.al = (T)al; L.cf = (T)cf;
}

template <typename T>
__device__ __forceinline__ T sqrt_t(T x) { return sqrt(x); }

// comoving unit vector n -> Eulerian (e, p) by the Lorentz boost (Sec. 3.2.2)
template <typename T>
__device__ __forceinline__ void boost_fwd(const Loc<T>& L, const T n[3], T& e, T p[3]) {
  T vn = L.v[0] * n[0] + L.v[1] * n[1] + L.v[2] * n[2];
  e = L.g * (T(1) + vn);
  T c = L.gg * vn + L.g;
  p[0] = n[0] + c * L.v[0];
  p[1] = n[1] + c * L.v[1];
  p[2] = n[2] + c * L.v[2];
}

// Eulerian (e, p) -> comoving of location L (inverse boost)
template <typename T>
__device__ __forceinline__ void boost_inv(const Loc<T>& L, T& e, T p[3]) {
  T vp = L.v[0] * p[0] + L.v[1] * p[1] + L.v[2] * p[2];
  T e2 = L.g * (e - vp);
  T c = L.gg * vp - L.g * e;
  p[0] += c * L.v[0];
  p[1] += c * L.v[1];
  p[2] += c * L.v[2];
  e = e2;
}

// Hamiltonian kick (Sec. 3.2.4) for the CFC metric with zero shift, on the
// Eulerian orthonormal components.  a = alpha_src/alpha_dst, b =
// (phi_src/phi_dst)^2.  Spatial step along `axis`: alpha e and the tangential
// phi^2 p_i are conserved, the normal component follows from the null
// condition with the root that vanishes continuously with the metric jump,
// and without a real root the normal covariant component is zeroed and the
// tangential ones rescaled (reflection).  Time step: phi^2 p conserved.
template <typename T>
__device__ __forceinline__ void kick(int axis, T a, T b, T& e, T p[3]) {
  if (axis == AX_TIME) {
    e *= b; p[0] *= b; p[1] *= b; p[2] *= b;
    return;
  }
  T pn = p[axis];
  T pt2 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (i != axis) pt2 += p[i] * p[i];
  T rad = a * a * pn * pn + (a * a - b * b) * pt2;
  e *= a;
  if (rad >= T(0)) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i != axis) p[i] *= b;
    p[axis] = (pn >= T(0) ? T(1) : T(-1)) * sqrt(rad);
  } else {
    T sc = e / sqrt(pt2);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (i != axis) p[i] *= sc;
    p[axis] = T(0);
  }
}

__device__ __forceinline__ double floor_t(double x) { return floor(x); }
__device__ __forceinline__ float floor_t(float x) { return floorf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double pow_t(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float pow_t(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double atan2_t(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float atan2_t(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }

// Mixed path: interpolation weights are rounded to multiples of 2^-17 so that
// w_L + w_R == 1 exactly and every product of three weights is exact in
// float64; the content deposits then conserve number to float64 round-off.
template <typename T>
__device__ __forceinline__ T qw(T w) { return w; }
template <>
__device__ __forceinline__ float qw<float>(float w) { return rintf(w * 131072.0f) * (1.0f / 131072.0f); }

// Full chain for source angle `ang`: comoving(src) -> Eulerian(src) -> kick
// -> rotation G (src triad -> dst triad; transposed if gT) -> comoving(dst),
// then the trilinear weights (Sec. 3.2, Eq. interpolation).
template <typename T>
__device__ void chain_weights(const Tables& tb, const T* s_mu, const Loc<T>& X, const Loc<T>& Y,
                              const double* G, int gT, int axis, int ang, Wt<T>& w) {
  const int j = ang / tb.n_ph, k = ang % tb.n_ph;
  T n[3];
  n[0] = s_mu[j];
  T sm = (T)tb.smu[j];
  n[1] = sm * (T)tb.cph[k];
  n[2] = sm * (T)tb.sph[k];
  T e, p[3];
  boost_fwd(X, n, e, p);
  T a = X.al / Y.al;
  T bq = (X.cf / Y.cf) * (X.cf / Y.cf);
  kick(axis, a, bq, e, p);
  if (G) {
    T q[3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
      q[m] = gT ? ((T)G[m] * p[0] + (T)G[3 + m] * p[1] + (T)G[6 + m] * p[2])
                : ((T)G[3 * m] * p[0] + (T)G[3 * m + 1] * p[1] + (T)G[3 * m + 2] * p[2]);
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
  }
  boost_inv(Y, e, p);
  const T rho = e;
  T mus = p[0] / e;
  mus = mus > T(1) ? T(1) : (mus < T(-1) ? T(-1) : mus);
  T phs = atan2_t(p[2], p[1]);
  if (phs < T(0)) phs += T(2 * kPi);
  // energy: eps* = rho eps_i, bracket eps_{i+m} <= eps* < eps_{i+m+1}
  T R = (T)tb.R;
  int m = (int)floor_t(log_t(rho) / log_t(R));
  T t = rho / pow_t(R, (T)m);
  T we = (t - T(1)) / (R - T(1));
  we = we < T(0) ? T(0) : (we > T(1) ? T(1) : we);
  // mu: linear between bracketing nodes; clamped outside [mu_0, mu_last]
  int jL;
  T wm;
  const int nmu = tb.n_mu;
  if (nmu == 1 || mus <= s_mu[0]) {
    jL = 0; wm = T(0);
  } else if (mus >= s_mu[nmu - 1]) {
    jL = nmu - 2; wm = T(1);
  } else {
    jL = 0;
    while (jL < nmu - 2 && s_mu[jL + 1] <= mus) ++jL;
    wm = (mus - s_mu[jL]) / (s_mu[jL + 1] - s_mu[jL]);
  }
  // Phi: linear in Phi between bracketing centres, periodic
  int kL;
  T wp;
  const int nph = tb.n_ph;
  if (nph == 1) {
    kL = 0; wp = T(0);
  } else {
    T u = phs / T(2 * kPi / nph) - T(0.5);
    T kf = floor_t(u);
    wp = u - kf;
    kL = ((int)kf) % nph;
    if (kL < 0) kL += nph;
  }
  w.wmu = qw(wm); w.wph = qw(wp); w.we = qw(we);
  w.jL = (short)jL; w.kL = (short)kL; w.m = (short)m; w.pad = 0;
}

// ---------------------------------------------------------------------------
// Bucketing of source angles by lower bracket (one warp per remap)
// ---------------------------------------------------------------------------
template <typename T>
__device__ void build_buckets(const Wt<T>* w, int nang, int nph, int nkeys, short* off, short* list, int* cnt) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < nkeys; k += 32) cnt[k] = 0;
  __syncwarp();
  for (int base = 0; base < nang; base += 32) {
    int bsrc = base + lane;
    bool act = bsrc < nang;
    unsigned mask = __ballot_sync(0xffffffffu, act);
    if (act) {
      int key = w[bsrc].jL * nph + w[bsrc].kL;
      unsigned peers = __match_any_sync(mask, key);
      if (lane == __ffs(peers) - 1) cnt[key] += __popc(peers);
    }
    __syncwarp();
  }
  // exclusive scan of the counts (chunked per lane, then a warp scan)
  int per = (nkeys + 31) / 32;
  int k0 = lane * per, k1 = min(k0 + per, nkeys);
  int loc = 0;
  for (int k = k0; k < k1; ++k) loc += cnt[k];
  int incl = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  int run = incl - loc;
  for (int k = k0; k < k1; ++k) {
    int c = cnt[k];
    off[k] = (short)run;
    run += c;
    cnt[k] = 0;
  }
  if (lane == 31) off[nkeys] = (short)incl;
  __syncwarp();
  for (int base = 0; base < nang; base += 32) {
    int bsrc = base + lane;
    bool act = bsrc < nang;
    unsigned mask = __ballot_sync(0xffffffffu, act);
    int key = 0;
    unsigned peers = 0;
    if (act) {
      key = w[bsrc].jL * nph + w[bsrc].kL;
      peers = __match_any_sync(mask, key);
      int rank = __popc(peers & ((1u << lane) - 1u));
      list[off[key] + cnt[key] + rank] = (short)bsrc;
    }
    __syncwarp();
    if (act && lane == __ffs(peers) - 1) cnt[key] += __popc(peers);
    __syncwarp();
  }
}

// Gather of one destination bin (ip, bp) of T[src]: sum over source angles in
// the candidate buckets, each with its clamped two-group energy split.
template <typename T, typename Acc>
__device__ __forceinline__ Acc gather_bin(int ip, int bp, int ne, int nang, int nmu, int nph, const T* src,
                                         const Wt<T>* w, const short* off, const short* list) {
  const int jp = bp / nph, kp = bp % nph;
  const int jmax = nmu >= 2 ? nmu - 2 : 0;
  Acc acc = Acc(0);
  int kc[2];
  int nk = 1;
  kc[0] = kp;
  if (nph > 1) { kc[1] = (kp - 1 + nph) % nph; nk = 2; }
  for (int dj = 0; dj < 2; ++dj) {
    int jL = jp - 1 + dj;
    if (jL < 0 || jL > jmax) continue;
    for (int dk = 0; dk < nk; ++dk) {
      int key = jL * nph + kc[dk];
      int e0 = off[key], e1 = off[key + 1];
      for (int q = e0; q < e1; ++q) {
        int bs = list[q];
        const Wt<T> W = w[bs];
        T wmu = (jp == W.jL ? T(1) - W.wmu : T(0)) + (jp == W.jL + 1 ? W.wmu : T(0));
        int kR = nph > 1 ? (W.kL + 1) % nph : W.kL;
        T wph = (kp == W.kL ? T(1) - W.wph : T(0)) + (kp == kR ? W.wph : T(0));
        Acc wa = (Acc)wmu * (Acc)wph;
        if (wa == Acc(0)) continue;
        int m = W.m;
        Acc se = Acc(0);
        // left target clamp(i+m) == ip, right target clamp(i+m+1) == ip
        int lo = (ip == 0) ? 0 : ip - m;
        int hi = (ip == ne - 1) ? ne - 1 : ip - m;
        lo = max(lo, 0); hi = min(hi, ne - 1);
        Acc wl = Acc(1) - (Acc)W.we;
        for (int i = lo; i <= hi; ++i) se += wl * (Acc)src[i * nang + bs];
        lo = (ip == 0) ? 0 : ip - m - 1;
        hi = (ip == ne - 1) ? ne - 1 : ip - m - 1;
        lo = max(lo, 0); hi = min(hi, ne - 1);
        for (int i = lo; i <= hi; ++i) se += (Acc)W.we * (Acc)src[i * nang + bs];
        acc += wa * se;
      }
    }
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Face construction (Sec. 3.3 faces, Sec. 3.3.4 boundaries)
// ---------------------------------------------------------------------------
// fidx: 0 inner radial face, 1 outer radial face, 2 lower polar face (2D) or
// the periodic polar face (column), 3 upper polar face (2D), 4 periodic
// azimuthal face.  Returns false if the face does not exist or has no area.
__device__ bool make_face(const Tables& tb, const State& st, int a, int b, int fidx, FaceDesc& F) {
  const int nr = tb.n_r;
  const int zone = b * nr + a;
  for (int k = 0; k < 4; ++k) { F.z[k] = -1; F.G[k] = nullptr; F.x[k] = 0.0; }
  const double* Gr = tb.slab ? nullptr : tb.G_r + 9 * b;
  if (fidx == 0 || fidx == 1) {
    F.axis = AX_R;
    int edge = fidx == 0 ? a : a + 1;
    F.area = tb.area_r[b * (nr + 1) + edge];
    if (F.area == 0.0) return false;
    if (edge == 0) { F.type = tb.slab ? F_OUTFLOW_Q : F_REFLECT_Q; F.own = 2; }
    else if (edge == nr) { F.type = F_OUTFLOW_P; F.own = 1; }
    else { F.type = F_INTERNAL; F.own = fidx == 0 ? 2 : 1; }
    for (int k = 0; k < 4; ++k) {
      int aa = edge - 2 + k;
      if (aa >= 0 && aa < nr) { F.z[k] = b * nr + aa; F.G[k] = Gr; F.x[k] = tb.r_c[aa]; }
    }
    F.xs = tb.r_e[edge];
  } else if (fidx == 2 || fidx == 3) {
    if (tb.slab) return false;
    F.axis = AX_TH;
    F.type = F_INTERNAL;
    const double rc = tb.r_c[a];
    if (tb.periodic_th) {
      if (fidx == 3) return false;
      F.area = tb.area_t[a];
      F.own = 3;
      const double d = tb.dth_col, thc = tb.th_c[0];
      for (int k = 0; k < 4; ++k) { F.z[k] = zone; F.G[k] = tb.G_t + 9 * k; F.x[k] = rc * (thc + (k - 1) * d); }
      F.xs = rc * (thc + 0.5 * d);
    } else {
      int edge = fidx == 2 ? b : b + 1;
      if (edge == 0 || edge == tb.n_th) return false;
      F.area = tb.area_t[edge * nr + a];
      F.own = fidx == 2 ? 2 : 1;
      for (int k = 0; k < 4; ++k) {
        int bb = edge - 2 + k;
        if (bb >= 0 && bb < tb.n_th) { F.z[k] = bb * nr + a; F.G[k] = tb.G_t + 9 * (4 * edge + k); F.x[k] = rc * tb.th_c[bb]; }
      }
      F.xs = rc * tb.th_e[edge];
    }
    if (F.area == 0.0) return false;
  } else {
    if (tb.slab) return false;
    F.axis = AX_PH;
    F.type = F_INTERNAL;
    F.own = 3;
    F.area = tb.area_p[zone];
    if (F.area == 0.0) return false;
    const double rs = tb.r_c[a] * sin(tb.th_c[b]);
    for (int k = 0; k < 4; ++k) { F.z[k] = zone; F.G[k] = tb.G_p + 9 * (4 * b + k); F.x[k] = rs * (k - 1) * tb.dphi; }
    F.xs = rs * 0.5 * tb.dphi;
  }
  F.dx = F.x[2] - F.x[1];
  // face background [R-12]: means of the two neighbours (velocities rotated
  // into the face triad); the present cell's values at boundaries, with the
  // normal velocity zeroed at a reflecting wall
  double vp[3] = {0, 0, 0}, vq[3] = {0, 0, 0};
  for (int side = 1; side <= 2; ++side) {
    int zz = F.z[side];
    if (zz < 0) continue;
    const double* v = st.v + 3 * zz;
    double* o = side == 1 ? vp : vq;
    const double* G = F.G[side];
    if (G) {
      for (int m = 0; m < 3; ++m) o[m] = G[3 * m] * v[0] + G[3 * m + 1] * v[1] + G[3 * m + 2] * v[2];
    } else {
      o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
    }
  }
  if (F.z[1] >= 0 && F.z[2] >= 0) {
    for (int m = 0; m < 3; ++m) F.v[m] = 0.5 * (vp[m] + vq[m]);
    F.al = 0.5 * (st.al[F.z[1]] + st.al[F.z[2]]);
    F.cf = 0.5 * (st.cf[F.z[1]] + st.cf[F.z[2]]);
  } else if (F.z[1] >= 0) {
    for (int m = 0; m < 3; ++m) F.v[m] = vp[m];
    F.al = st.al[F.z[1]]; F.cf = st.cf[F.z[1]];
  } else {
    for (int m = 0; m < 3; ++m) F.v[m] = vq[m];
    F.al = st.al[F.z[2]]; F.cf = st.cf[F.z[2]];
    if (F.type == F_REFLECT_Q) F.v[F.axis] = 0.0;
  }
  return true;
}

__device__ __forceinline__ int nkeys_of(const Tables& tb) { return (tb.n_mu >= 2 ? tb.n_mu - 1 : 1) * tb.n_ph; }

// Shared-memory carve-up of the flux kernel.
template <typename T>
struct FluxSmem {
  double* dN;      // [ns][ne][nang]
  T* src;          // [ne][nang]
  T* g;            // [4][ne][nang]
  Wt<T>* W;        // [6][nang]
  short* off;      // [6][nkeys + 1]
  short* list;     // [6][nang]
  int* cnt;        // [6][nkeys]
  T* u0s;          // [nang] face
  T* vns;          // [nang]
  T* rowJ;         // [ne]
  T* kaS; T* ksS; T* feS; T* wP; T* wQ;  // [ne]
  T* mu;           // [nmu]
  double* zu0;     // [nang] own zone u^0
  double* zrow;    // [ns][ne][5] collision moment partials
  double* red;     // [kWarps * 2]
  double* tally;   // [ns][2] outflow N, E of this zone
  FaceDesc* F;
};

template <typename T>
__host__ __device__ size_t flux_smem_layout(int ns, int ne, int nang, int nmu, int nph, FluxSmem<T>* s, unsigned char* base) {
  size_t o = 0;
  const int nbin = ne * nang;
  const int nkeys = (nmu >= 2 ? nmu - 1 : 1) * nph;
#define BT_TAKE(ptr, type, count)                              \
  do {                                                         \
    o = (o + 15) & ~size_t(15);                                \
    if (s) s->ptr = reinterpret_cast<type*>(base + o);         \
    o += sizeof(type) * (size_t)(count);                       \
  } while (0)
  BT_TAKE(dN, double, (size_t)ns * nbin);
  BT_TAKE(zu0, double, nang);
  BT_TAKE(zrow, double, (size_t)ns * ne * 5);
  BT_TAKE(red, double, kWarps * 2);
  BT_TAKE(tally, double, ns * 2);
  BT_TAKE(src, T, nbin);
  BT_TAKE(g, T, 4 * nbin);
  BT_TAKE(W, Wt<T>, 6 * nang);
  BT_TAKE(u0s, T, nang);
  BT_TAKE(vns, T, nang);
  BT_TAKE(rowJ, T, ne);
  BT_TAKE(kaS, T, ne);
  BT_TAKE(ksS, T, ne);
  BT_TAKE(feS, T, ne);
  BT_TAKE(wP, T, ne);
  BT_TAKE(wQ, T, ne);
  BT_TAKE(mu, T, nmu);
  BT_TAKE(off, short, 6 * (nkeys + 1));
  BT_TAKE(list, short, 6 * nang);
  BT_TAKE(cnt, int, 6 * nkeys);
  BT_TAKE(F, FaceDesc, 1);
#undef BT_TAKE
  return (o + 15) & ~size_t(15);
}

template <typename T>
__device__ __forceinline__ T mc_limiter(T a, T b) {
  if (a * b <= T(0)) return T(0);
  T s = a > T(0) ? T(1) : T(-1);
  T x = fabs(T(2) * a), y = fabs(T(2) * b), z = T(0.5) * fabs(a + b);
  T m = x < y ? x : y;
  m = m < z ? m : z;
  return s * m;
}

__device__ __forceinline__ double block_sum2(double v0, double v1, double* red, double& out1) {
  // deterministic block reduction of two values
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_down_sync(0xffffffffu, v0, o);
    v1 += __shfl_down_sync(0xffffffffu, v1, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[2 * w] = v0; red[2 * w + 1] = v1; }
  __syncthreads();
  double s0 = 0.0, s1 = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWarps; ++i) { s0 += red[2 * i]; s1 += red[2 * i + 1]; }
  }
  __syncthreads();
  out1 = s1;
  return s0;
}

// ---------------------------------------------------------------------------
// Fused face fluxes + collision of one zone (Sec. 3.3, 3.5, 3.4)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) k_flux_collide(Tables tb, State st, double dt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FluxSmem<T> S;
  flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, &S, smem_raw);
  const int zone = blockIdx.x;
  const int a = zone % tb.n_r, b = zone / tb.n_r;
  const int NE = tb.n_e, NA = tb.n_ang, NS = tb.n_s, NPH = tb.n_ph, NMU = tb.n_mu;
  const int nbin = NE * NA;
  const int nkeys = nkeys_of(tb);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const T* fin = reinterpret_cast<const T*>(st.f);
  T* fout = reinterpret_cast<T*>(st.f_next);

  for (int q = tid; q < NS * nbin; q += kThreads) S.dN[q] = 0.0;
  for (int q = tid; q < NMU; q += kThreads) S.mu[q] = (T)tb.mu[q];
  for (int q = tid; q < NS * 2; q += kThreads) S.tally[q] = 0.0;
  __syncthreads();

  const int nface = tb.slab ? 2 : 5;
  for (int fidx = 0; fidx < nface; ++fidx) {
    if (tid == 0) {
      bool ok = make_face(tb, st, a, b, fidx, *S.F);
      if (!ok) S.F->type = -1;
    }
    __syncthreads();
    const FaceDesc& F = *S.F;
    if (F.type < 0) { __syncthreads(); continue; }

    // --- weights of the six remaps: slots 0..3 -> face, face -> slot 1, face -> slot 2
    {
      Loc<T> Ls;
      make_loc(Ls, F.v, F.al, F.cf);
      for (int q = tid; q < 6 * NA; q += kThreads) {
        int r = q / NA, ang = q % NA;
        int slot = r < 4 ? r : r - 3;
        bool need = r < 4 ? (F.z[slot] >= 0) : ((r == 4 && (F.own & 1)) || (r == 5 && (F.own & 2)));
        if (!need) continue;
        int zz = F.z[slot];
        Loc<T> Lc;
        make_loc(Lc, st.v + 3 * zz, st.al[zz], st.cf[zz]);
        Wt<T> w;
        if (r < 4) chain_weights(tb, S.mu, Lc, Ls, F.G[slot], 0, F.axis, ang, w);
        else chain_weights(tb, S.mu, Ls, Lc, F.G[slot], 1, F.axis, ang, w);
        S.W[r * NA + ang] = w;
      }
      // face bins: Eulerian energy factor and normal coordinate velocity
      for (int ang = tid; ang < NA; ang += kThreads) {
        const int j = ang / NPH, k = ang % NPH;
        T n[3] = {S.mu[j], (T)tb.smu[j] * (T)tb.cph[k], (T)tb.smu[j] * (T)tb.sph[k]};
        T e, p[3];
        boost_fwd(Ls, n, e, p);
        S.u0s[ang] = e;
        S.vns[ang] = Ls.al / (Ls.cf * Ls.cf) * p[F.axis] / e;
      }
    }
    __syncthreads();
    if (warp < 6) {
      int r = warp;
      int slot = r < 4 ? r : r - 3;
      bool need = r < 4 ? (F.z[slot] >= 0) : ((r == 4 && (F.own & 1)) || (r == 5 && (F.own & 2)));
      if (need) build_buckets(S.W + r * NA, NA, NPH, nkeys, S.off + r * (nkeys + 1), S.list + r * NA, S.cnt + r * nkeys);
    }
    __syncthreads();

    const T c6s = (T)pow(F.cf, 6.0);
    for (int s = 0; s < NS; ++s) {
      // face opacities and flux-switch weights per group [R-10, R-12b]
      if (F.type == F_INTERNAL) {
        for (int i = tid; i < NE; i += kThreads) {
          size_t oP = ((size_t)s * tb.n_zone + F.z[1]) * NE + i;
          size_t oQ = ((size_t)s * tb.n_zone + F.z[2]) * NE + i;
          double kaP = st.ka[oP], kaQ = st.ka[oQ], ksP = st.ks[oP], ksQ = st.ks[oQ];
          S.kaS[i] = (T)(0.5 * (kaP + kaQ));
          S.ksS[i] = (T)(0.5 * (ksP + ksQ));
          S.feS[i] = (T)(0.5 * (st.fe[oP] + st.fe[oQ]));
          S.wP[i] = exp_t((T)(-(kaP + ksP)) * (T)F.dx);
          S.wQ[i] = exp_t((T)(-(kaQ + ksQ)) * (T)F.dx);
        }
      }
      // stencil contents remapped into the face frame: g_k = T_{k->s}[n_k]
      for (int slot = 0; slot < 4; ++slot) {
        const int zz = F.z[slot];
        if (zz < 0) continue;
        Loc<T> Lc;
        make_loc(Lc, st.v + 3 * zz, st.al[zz], st.cf[zz]);
        const T c6 = (T)pow(st.cf[zz], 6.0);
        const T* fz = fin + ((size_t)s * tb.n_zone + zz) * nbin;
        for (int q = tid; q < nbin; q += kThreads) {
          int i = q / NA, ang = q % NA;
          int j = ang / NPH, k = ang % NPH;
          T nv = Lc.v[0] * S.mu[j] + (Lc.v[1] * (T)tb.cph[k] + Lc.v[2] * (T)tb.sph[k]) * (T)tb.smu[j];
          T u0 = Lc.g * (T(1) + nv);
          S.src[q] = c6 * u0 * (T)tb.dGam[i] * (T)tb.dOm[ang] * fz[q];
        }
        __syncthreads();
        T* gk = S.g + slot * nbin;
        const Wt<T>* W = S.W + slot * NA;
        const short* off = S.off + slot * (nkeys + 1);
        const short* lst = S.list + slot * NA;
        for (int q = tid; q < nbin; q += kThreads) {
          int ip = q / NA, bp = q % NA;
          T d = gather_bin<T, T>(ip, bp, NE, NA, NMU, NPH, S.src, W, off, lst);
          gk[q] = d / (c6s * S.u0s[bp] * (T)tb.dGam[ip] * (T)tb.dOm[bp]);
        }
        __syncthreads();
      }
      // Lax-Wendroff half step with implicit collision: J per group (one warp per row)
      const T hdt = T(0.5) * (T)dt;
      if (F.type == F_INTERNAL) {
        for (int i = warp; i < NE; i += kWarps) {
          T sr = T(0), s1 = T(0);
          const T ka = S.kaS[i], ks = S.ksS[i], fe = S.feS[i];
          for (int ang = lane; ang < NA; ang += 32) {
            int q = i * NA + ang;
            T g1 = S.g[nbin + q], g2 = S.g[2 * nbin + q];
            T tau = hdt * (T)F.al / S.u0s[ang];
            T r = T(0.5) * (g1 + g2) - hdt * S.vns[ang] * (g2 - g1) / (T)F.dx + tau * ka * fe;
            T D = T(1) + (ka + ks) * tau;
            T dom = (T)tb.dOm[ang];
            sr += dom * r / D;
            s1 += dom * (T(1) + ka * tau) / D;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_down_sync(0xffffffffu, sr, o);
            s1 += __shfl_down_sync(0xffffffffu, s1, o);
          }
          if (lane == 0) S.rowJ[i] = sr / s1;
        }
        __syncthreads();
      }
      // interface state (blend of LW and MC upwind) and flux content per face bin
      for (int q = tid; q < nbin; q += kThreads) {
        int i = q / NA, ang = q % NA;
        T vn = S.vns[ang];
        T fs;
        if (F.type == F_INTERNAL) {
          T g0 = S.g[q], g1 = S.g[nbin + q], g2 = S.g[2 * nbin + q], g3 = S.g[3 * nbin + q];
          const T ka = S.kaS[i], ks = S.ksS[i], fe = S.feS[i];
          T tau = hdt * (T)F.al / S.u0s[ang];
          T r = T(0.5) * (g1 + g2) - hdt * vn * (g2 - g1) / (T)F.dx + tau * ka * fe;
          T D = T(1) + (ka + ks) * tau;
          T flw = (r + ks * tau * S.rowJ[i]) / D;
          T fu, w;
          if (vn >= T(0)) {
            T sl = T(0);
            if (F.z[0] >= 0) sl = mc_limiter((g1 - g0) / (T)(F.x[1] - F.x[0]), (g2 - g1) / (T)(F.x[2] - F.x[1]));
            fu = g1 + sl * (T)(F.xs - F.x[1]);
            w = S.wP[i];
          } else {
            T sl = T(0);
            if (F.z[3] >= 0) sl = mc_limiter((g2 - g1) / (T)(F.x[2] - F.x[1]), (g3 - g2) / (T)(F.x[3] - F.x[2]));
            fu = g2 + sl * (T)(F.xs - F.x[2]);
            w = S.wQ[i];
          }
          fs = (T(1) - w) * flw + w * fu;
        } else if (F.type == F_OUTFLOW_P) {
          fs = vn >= T(0) ? S.g[nbin + q] : T(0);
        } else if (F.type == F_OUTFLOW_Q) {
          fs = vn < T(0) ? S.g[2 * nbin + q] : T(0);
        } else {  // reflecting wall at rest
          int j = ang / NPH, k = ang % NPH;
          int qm = i * NA + (NMU - 1 - j) * NPH + k;
          fs = vn < T(0) ? S.g[2 * nbin + q] : S.g[2 * nbin + qm];
        }
        S.src[q] = (T)dt * (T)F.area * c6s * S.u0s[ang] * vn * (T)tb.dGam[i] * (T)tb.dOm[ang] * fs;
      }
      __syncthreads();
      // outflow tallies (number and energy at infinity)
      if (F.type == F_OUTFLOW_P || F.type == F_OUTFLOW_Q) {
        double sg = F.type == F_OUTFLOW_P ? 1.0 : -1.0;
        double tn = 0.0, te = 0.0;
        for (int q = tid; q < nbin; q += kThreads) {
          int i = q / NA, ang = q % NA;
          double c = sg * (double)S.src[q];
          tn += c;
          te += c * F.al * tb.eps[i] * (double)S.u0s[ang];
        }
        double te_sum;
        double tn_sum = block_sum2(tn, te, S.red, te_sum);
        if (tid == 0) { S.tally[2 * s] += tn_sum; S.tally[2 * s + 1] += te_sum; }
      }
      // deposits into this zone: dN -= T_{s->P}[F] (own P), dN += T_{s->Q}[F] (own Q)
      double* dNs = S.dN + (size_t)s * nbin;
      for (int q = tid; q < nbin; q += kThreads) {
        int ip = q / NA, bp = q % NA;
        double acc = 0.0;
        if (F.own & 1) acc -= gather_bin<T, double>(ip, bp, NE, NA, NMU, NPH, S.src, S.W + 4 * NA, S.off + 4 * (nkeys + 1), S.list + 4 * NA);
        if (F.own & 2) acc += gather_bin<T, double>(ip, bp, NE, NA, NMU, NPH, S.src, S.W + 5 * NA, S.off + 5 * (nkeys + 1), S.list + 5 * NA);
        dNs[q] += acc;
      }
      __syncthreads();
    }
  }

  // --- implicit collision per (species, group) (Sec. 3.5) and moments (Eq. hydrosource)
  const double alz = st.al[zone], c6z = pow(st.cf[zone], 6.0), volz = tb.vol[zone];
  {
    const double* v = st.v + 3 * zone;
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    double gz = 1.0 / sqrt(1.0 - v2);
    for (int ang = tid; ang < NA; ang += kThreads) {
      int j = ang / NPH, k = ang % NPH;
      double nv = v[0] * tb.mu[j] + (v[1] * tb.cph[k] + v[2] * tb.sph[k]) * tb.smu[j];
      S.zu0[ang] = gz * (1.0 + nv);
    }
  }
  __syncthreads();
  for (int row = warp; row < NS * NE; row += kWarps) {
    const int s = row / NE, i = row % NE;
    const size_t oz = ((size_t)s * tb.n_zone + zone) * NE + i;
    const double ka = st.ka[oz], ks = st.ks[oz], fe = st.fe[oz];
    const T* fz = fin + ((size_t)s * tb.n_zone + zone) * nbin + (size_t)i * NA;
    const double* dn = S.dN + (size_t)s * nbin + (size_t)i * NA;
    const double dg = tb.dGam[i];
    double sr = 0.0, s1 = 0.0;
    for (int ang = lane; ang < NA; ang += 32) {
      double u0 = S.zu0[ang];
      double tau = alz * dt / u0;
      double fst = (double)fz[ang] + dn[ang] / (c6z * volz * u0 * dg * tb.dOm[ang]);
      double r = fst + tau * ka * fe;
      double D = 1.0 + (ka + ks) * tau;
      sr += tb.dOm[ang] * r / D;
      s1 += tb.dOm[ang] * (1.0 + ka * tau) / D;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const double J = sr / s1;
    double mN = 0.0, mE = 0.0, mP0 = 0.0, mP1 = 0.0, mP2 = 0.0;
    int bad = 0;
    T* fo = fout + ((size_t)s * tb.n_zone + zone) * nbin + (size_t)i * NA;
    for (int ang = lane; ang < NA; ang += 32) {
      const int j = ang / NPH, k = ang % NPH;
      double u0 = S.zu0[ang];
      double tau = alz * dt / u0;
      double fst = (double)fz[ang] + dn[ang] / (c6z * volz * u0 * dg * tb.dOm[ang]);
      double r = fst + tau * ka * fe;
      double D = 1.0 + (ka + ks) * tau;
      double fn = (r + ks * tau * J) / D;
      T fw = (T)fn;
      fo[ang] = fw;
      bad |= !isfinite(fn);
      double dc = c6z * u0 * dg * tb.dOm[ang] * ((double)fw - fst) / dt;
      mN += dc;
      double de = dc * tb.eps[i];
      mE += de;
      mP0 += de * tb.mu[j];
      mP1 += de * tb.smu[j] * tb.cph[k];
      mP2 += de * tb.smu[j] * tb.sph[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mN += __shfl_xor_sync(0xffffffffu, mN, o);
      mE += __shfl_xor_sync(0xffffffffu, mE, o);
      mP0 += __shfl_xor_sync(0xffffffffu, mP0, o);
      mP1 += __shfl_xor_sync(0xffffffffu, mP1, o);
      mP2 += __shfl_xor_sync(0xffffffffu, mP2, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      double* zr = S.zrow + (size_t)row * 5;
      zr[0] = mN; zr[1] = mE; zr[2] = mP0; zr[3] = mP1; zr[4] = mP2;
      if (bad) st.flag[0] = 1;
    }
  }
  __syncthreads();
  for (int s = tid; s < NS; s += kThreads) {
    double m[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < NE; ++i)
      for (int c = 0; c < 5; ++c) m[c] += S.zrow[((size_t)s * NE + i) * 5 + c];
    size_t o = (size_t)s * tb.n_zone + zone;
    st.mom_N[o] = m[0];
    st.mom_E[o] = m[1];
    st.mom_P[3 * o] = m[2]; st.mom_P[3 * o + 1] = m[3]; st.mom_P[3 * o + 2] = m[4];
    st.out_N[o] = S.tally[2 * s];
    st.out_E[o] = S.tally[2 * s + 1];
  }
  if (tid == 0) {
    // Q_Ye = -(dN_nue - dN_nuebar) / h^3 (Eq. hydrosource)
    double q = 0.0;
    for (int s = 0; s < NS; ++s) {
      int kind = tb.species_kind[s];
      if (kind != 0 && kind != 1) continue;
      double m = 0.0;
      for (int i = 0; i < NE; ++i) m += S.zrow[((size_t)s * NE + i) * 5];
      q += kind == 0 ? -m : m;
    }
    st.qye[zone] = q * st.phase_norm;
  }
}

// ---------------------------------------------------------------------------
// Time remap T_{n->n+1} of every zone (Sec. 3.2): old frames -> new frames
// ---------------------------------------------------------------------------
template <typename T>
struct RemapSmem {
  T* src; T* mu; Wt<T>* W; short* off; short* list; int* cnt;
};

template <typename T>
__host__ __device__ size_t remap_smem_layout(int ne, int nang, int nmu, int nph, RemapSmem<T>* s, unsigned char* base) {
  size_t o = 0;
  const int nkeys = (nmu >= 2 ? nmu - 1 : 1) * nph;
#define BT_TAKE(ptr, type, count)                              \
  do {                                                         \
    o = (o + 15) & ~size_t(15);                                \
    if (s) s->ptr = reinterpret_cast<type*>(base + o);         \
    o += sizeof(type) * (size_t)(count);                       \
  } while (0)
  BT_TAKE(src, T, (size_t)ne * nang);
  BT_TAKE(mu, T, nmu);
  BT_TAKE(W, Wt<T>, nang);
  BT_TAKE(off, short, nkeys + 1);
  BT_TAKE(list, short, nang);
  BT_TAKE(cnt, int, nkeys);
#undef BT_TAKE
  return (o + 15) & ~size_t(15);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_time_remap(Tables tb, State st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RemapSmem<T> S;
  remap_smem_layout<T>(tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, &S, smem_raw);
  const int zone = blockIdx.x;
  const int NE = tb.n_e, NA = tb.n_ang, NPH = tb.n_ph, NMU = tb.n_mu;
  const int nbin = NE * NA, nkeys = nkeys_of(tb);
  const int tid = threadIdx.x;
  for (int q = tid; q < NMU; q += kThreads) S.mu[q] = (T)tb.mu[q];
  __syncthreads();
  Loc<T> X, Y;
  make_loc(X, st.v_old + 3 * zone, st.al_old[zone], st.cf_old[zone]);
  make_loc(Y, st.v + 3 * zone, st.al[zone], st.cf[zone]);
  for (int ang = tid; ang < NA; ang += kThreads) chain_weights(tb, S.mu, X, Y, nullptr, 0, AX_TIME, ang, S.W[ang]);
  __syncthreads();
  if (tid < 32) build_buckets(S.W, NA, NPH, nkeys, S.off, S.list, S.cnt);
  __syncthreads();
  const T c6x = (T)pow(st.cf_old[zone], 6.0), c6y = (T)pow(st.cf[zone], 6.0);
  T* f = reinterpret_cast<T*>(st.f);
  for (int s = 0; s < tb.n_s; ++s) {
    T* fz = f + ((size_t)s * tb.n_zone + zone) * nbin;
    for (int q = tid; q < nbin; q += kThreads) {
      int i = q / NA, ang = q % NA;
      int j = ang / NPH, k = ang % NPH;
      T nv = X.v[0] * S.mu[j] + (X.v[1] * (T)tb.cph[k] + X.v[2] * (T)tb.sph[k]) * (T)tb.smu[j];
      S.src[q] = c6x * X.g * (T(1) + nv) * (T)tb.dGam[i] * (T)tb.dOm[ang] * fz[q];
    }
    __syncthreads();
    for (int q = tid; q < nbin; q += kThreads) {
      int ip = q / NA, bp = q % NA;
      int j = bp / NPH, k = bp % NPH;
      double d = gather_bin<T, double>(ip, bp, NE, NA, NMU, NPH, S.src, S.W, S.off, S.list);
      T nv = Y.v[0] * S.mu[j] + (Y.v[1] * (T)tb.cph[k] + Y.v[2] * (T)tb.sph[k]) * (T)tb.smu[j];
      T u0 = Y.g * (T(1) + nv);
      fz[q] = (T)(d / ((double)c6y * (double)u0 * tb.dGam[ip] * tb.dOm[bp]));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Diagnostics: totals, outflow accumulation, Courant rate, J/H/K
// ---------------------------------------------------------------------------
// per-zone partial totals: red[(s*nz + zone)*2 + {0,1}] = (N, E)
template <typename T>
__global__ void __launch_bounds__(kThreads) k_zone_totals(Tables tb, State st) {
  __shared__ double red[kWarps * 2];
  const int zone = blockIdx.x;
  const int NE = tb.n_e, NA = tb.n_ang, NPH = tb.n_ph;
  const int nbin = NE * NA;
  const T* f = reinterpret_cast<const T*>(st.f);
  const double* v = st.v + 3 * zone;
  const double gz = 1.0 / sqrt(1.0 - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
  const double c6 = pow(st.cf[zone], 6.0), al = st.al[zone], vol = tb.vol[zone];
  for (int s = 0; s < tb.n_s; ++s) {
    const T* fz = f + ((size_t)s * tb.n_zone + zone) * nbin;
    double sn = 0.0, se = 0.0;
    for (int q = threadIdx.x; q < nbin; q += kThreads) {
      int i = q / NA, ang = q % NA;
      int j = ang / NPH, k = ang % NPH;
      double u0 = gz * (1.0 + v[0] * tb.mu[j] + (v[1] * tb.cph[k] + v[2] * tb.sph[k]) * tb.smu[j]);
      double c = vol * c6 * u0 * tb.dGam[i] * tb.dOm[ang] * (double)fz[q];
      sn += c;
      se += c * al * tb.eps[i] * u0;
    }
    double e_sum;
    double n_sum = block_sum2(sn, se, red, e_sum);
    if (threadIdx.x == 0) {
      st.red[((size_t)s * tb.n_zone + zone) * 2] = n_sum;
      st.red[((size_t)s * tb.n_zone + zone) * 2 + 1] = e_sum;
    }
  }
}

// Neumaier-compensated sum of `n` strided values, one CTA per output.
__device__ void comp_add(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

// out[o] = sum_{zone} in[(o/2)*nz*2 + zone*2 + o%2]  for o in [0, 2*n_s)
__global__ void __launch_bounds__(kThreads) k_reduce_pairs(const double* in, int nz, double* out, int accumulate) {
  __shared__ double ss[kThreads], cc[kThreads];
  const int o = blockIdx.x;
  const int s = o / 2, c = o % 2;
  double sum = 0.0, comp = 0.0;
  for (int z = threadIdx.x; z < nz; z += kThreads) comp_add(sum, comp, in[((size_t)s * nz + z) * 2 + c]);
  ss[threadIdx.x] = sum;
  cc[threadIdx.x] = comp;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int t = 0; t < kThreads; ++t) { comp_add(S, C, ss[t]); C += cc[t]; }
    if (accumulate) {
      // out holds (sum, compensation) pairs: [o] value, [2*n_s*? ] handled by caller layout
      double prev = out[2 * o], prevc = out[2 * o + 1];
      double t = prev;
      comp_add(t, prevc, S + C);
      out[2 * o] = t;
      out[2 * o + 1] = prevc;
    } else {
      out[o] = S + C;
    }
  }
}

// pack per-zone outflow (N, E) pairs into the reduction scratch
__global__ void k_pack_outflow(Tables tb, State st) {
  size_t n = (size_t)tb.n_s * tb.n_zone;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    st.red[2 * q] = st.out_N[q];
    st.red[2 * q + 1] = st.out_E[q];
  }
}

// Courant rate (C-14 reading): max over zones and bins of sum over the zone's
// faces of max(0, outward coordinate velocity) dA/dV.
__global__ void __launch_bounds__(kThreads) k_max_rate(Tables tb, State st, unsigned long long* out) {
  __shared__ FaceDesc F;
  __shared__ double rate[kMaxAng];
  __shared__ double red[kWarps];
  const int zone = blockIdx.x;
  const int a = zone % tb.n_r, b = zone / tb.n_r;
  const int NA = tb.n_ang, NPH = tb.n_ph;
  for (int q = threadIdx.x; q < NA; q += kThreads) rate[q] = 0.0;
  const int nface = tb.slab ? 2 : 5;
  Loc<double> L;
  make_loc(L, st.v + 3 * zone, st.al[zone], st.cf[zone]);
  const double vol = tb.vol[zone];
  for (int fidx = 0; fidx < nface; ++fidx) {
    __syncthreads();
    if (threadIdx.x == 0) { if (!make_face(tb, st, a, b, fidx, F)) F.type = -1; }
    __syncthreads();
    if (F.type < 0) continue;
    for (int ang = threadIdx.x; ang < NA; ang += kThreads) {
      int j = ang / NPH, k = ang % NPH;
      double n[3] = {tb.mu[j], tb.smu[j] * tb.cph[k], tb.smu[j] * tb.sph[k]};
      double e, p[3];
      boost_fwd(L, n, e, p);
      for (int side = 1; side <= 2; ++side) {
        if (!(F.own & side)) continue;
        const double* G = F.G[side];
        double pn = G ? (G[3 * F.axis] * p[0] + G[3 * F.axis + 1] * p[1] + G[3 * F.axis + 2] * p[2]) : p[F.axis];
        double vel = (side == 1 ? 1.0 : -1.0) * L.al / (L.cf * L.cf) * pn / e;
        if (vel > 0.0) rate[ang] += vel * F.area / vol;
      }
    }
  }
  __syncthreads();
  double m = 0.0;
  for (int q = threadIdx.x; q < NA; q += kThreads) m = fmax(m, rate[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < kWarps; ++w) mm = fmax(mm, red[w]);
    atomicMax(out, (unsigned long long)__double_as_longlong(mm));
  }
}

template <typename T>
__global__ void k_jhk(Tables tb, State st, double* J, double* H, double* K) {
  size_t nrow = (size_t)tb.n_s * tb.n_zone * tb.n_e;
  const int NA = tb.n_ang, NPH = tb.n_ph;
  const T* f = reinterpret_cast<const T*>(st.f);
  for (size_t row = blockIdx.x * (size_t)blockDim.x + threadIdx.x; row < nrow; row += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(row % tb.n_e);
    const T* fr = f + row * NA;
    double sj = 0.0, sh = 0.0, sk = 0.0;
    for (int ang = 0; ang < NA; ++ang) {
      double mu = tb.mu[ang / NPH];
      double c = tb.dOm[ang] * (double)fr[ang] * tb.eps[i] * tb.dGam[i] / (4.0 * kPi);
      sj += c; sh += c * mu; sk += c * mu * mu;
    }
    J[row] = sj; H[row] = sh; K[row] = sk;
  }
}

template <typename T>
int launch_flux_t(const Tables& tb, const State& st, double dt, cudaStream_t s) {
  size_t sm = flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr);
  cudaError_t e = cudaFuncSetAttribute(k_flux_collide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  k_flux_collide<T><<<tb.n_zone, kThreads, sm, s>>>(tb, st, dt);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_remap_t(const Tables& tb, const State& st, cudaStream_t s) {
  size_t sm = remap_smem_layout<T>(tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr);
  cudaError_t e = cudaFuncSetAttribute(k_time_remap<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  k_time_remap<T><<<tb.n_zone, kThreads, sm, s>>>(tb, st);
  return (int)cudaGetLastError();
}

}  // namespace

size_t flux_smem_bytes(const Tables& tb, int mixed) {
  return mixed ? flux_smem_layout<float>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr)
               : flux_smem_layout<double>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr);
}
size_t remap_smem_bytes(const Tables& tb, int mixed) {
  return mixed ? remap_smem_layout<float>(tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr)
               : remap_smem_layout<double>(tb.n_e, tb.n_ang, tb.n_mu, tb.n_ph, nullptr, nullptr);
}
int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int launch_flux_collide(const Tables& tb, const State& st, double dt, int mixed, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return mixed ? launch_flux_t<float>(tb, st, dt, s) : launch_flux_t<double>(tb, st, dt, s);
}

int launch_time_remap(const Tables& tb, const State& st, int mixed, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  return mixed ? launch_remap_t<float>(tb, st, s) : launch_remap_t<double>(tb, st, s);
}

int launch_totals(const Tables& tb, const State& st, int mixed, double* d_out, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (mixed) k_zone_totals<float><<<tb.n_zone, kThreads, 0, s>>>(tb, st);
  else k_zone_totals<double><<<tb.n_zone, kThreads, 0, s>>>(tb, st);
  k_reduce_pairs<<<2 * tb.n_s, kThreads, 0, s>>>(st.red, tb.n_zone, d_out, 0);
  return (int)cudaGetLastError();
}

int launch_accumulate_outflow(const Tables& tb, const State& st, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  k_pack_outflow<<<64, kThreads, 0, s>>>(tb, st);
  k_reduce_pairs<<<2 * tb.n_s, kThreads, 0, s>>>(st.red, tb.n_zone, st.acc, 1);
  return (int)cudaGetLastError();
}

int launch_max_rate(const Tables& tb, const State& st, double* d_rate, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(d_rate, 0, sizeof(double), s);
  k_max_rate<<<tb.n_zone, kThreads, 0, s>>>(tb, st, reinterpret_cast<unsigned long long*>(d_rate));
  return (int)cudaGetLastError();
}

int launch_jhk(const Tables& tb, const State& st, int mixed, double* J, double* H, double* K, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  size_t nrow = (size_t)tb.n_s * tb.n_zone * tb.n_e;
  int blocks = (int)((nrow + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (mixed) k_jhk<float><<<blocks, 256, 0, s>>>(tb, st, J, H, K);
  else k_jhk<double><<<blocks, 256, 0, s>>>(tb, st, J, H, K);
  return (int)cudaGetLastError();
}

int launch_check_finite(const Tables&, const State&, int, void*) { return 0; }

}  // namespace bt
