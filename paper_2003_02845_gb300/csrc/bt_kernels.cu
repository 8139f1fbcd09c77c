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
#include "bt_tc.cuh"

namespace bt {

namespace {

constexpr int kThreads = 256;   // block size of the non-tuned kernels
constexpr int kWarps = kThreads / 32;
constexpr int kMaxWarps = 16;    // largest tuned block: 512 threads
constexpr double kPi = 3.14159265358979323846;

// weights of one source angle for one remap
template <typename T>
struct Wt {
  T wmu, wph, we;
  short jL, kL, m, pad;
};

struct FaceDesc {
  int type, axis, own;  // own: 1 = P, 2 = Q, 3 = both (periodic face)
  int bc;               // open face at theta_max: incoming bins take State::fbc
  int addP, addQ;       // local time stepping: add to the side's deposit row (its step began earlier)
  int z[4];             // zone of stencil slot k (P-1, P, Q, Q+1), -1 absent
  const double* G[4];   // rotation: slot k triad -> face triad (row-major 3x3)
  double x[4], xs, dx, area;
  double v[3], al, cf;  // face background
};

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
__device__ __forceinline__ double atan2_t(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float atan2_t(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float exp_t(float x) { return expf(x); }

// constants of the energy bracket on a grid of ratio R, formed once per
// thread: log R, 1/log R, 1/(R-1)
template <typename T>
struct EBr {
  T lR, rlR, rRm1;
};
template <typename T>
__device__ __forceinline__ EBr<T> make_ebr(T R) {
  EBr<T> k;
  k.lR = log_t(R);
  k.rlR = T(1) / k.lR;
  k.rRm1 = T(1) / (R - T(1));
  return k;
}

// Full chain for source angle `ang`: comoving(src) -> Eulerian(src) -> kick
// -> rotation G (src triad -> dst triad; transposed if gT) -> comoving(dst),
// then the trilinear weights (Sec. 3.2, Eq. interpolation).
template <typename T>
__device__ void chain_weights_dir(const Tables& tb, const T* s_mu, const T* n, const Loc<T>& X, const Loc<T>& Y,
                                  const T* G, int gT, int axis, const EBr<T>& K, Wt<T>& w) {
  T e, p[3];
  boost_fwd(X, n, e, p);
  // the metric ratios by correctly rounded divisions: where the metric is the
  // same on both sides (periodic images, equal neighbours, flat regions)
  // they are exactly 1.  A reciprocal then a product can round to 1 - ulp,
  // and for a direction tangent to the face (normal component 0, e.g. the
  // pole cells of a Gauss-Lobatto grid at polar and azimuthal faces) the
  // kick's normal component sqrt(a^2 - b^2) |p_t| would then be sqrt(ulp)
  // instead of 0.
  const T a = X.al / Y.al;
  const T cr = X.cf / Y.cf;
  const T bq = cr * cr;
  kick(axis, a, bq, e, p);
  if (G) {
    T q[3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
      q[m] = gT ? (G[m] * p[0] + G[3 + m] * p[1] + G[6 + m] * p[2])
                : (G[3 * m] * p[0] + G[3 * m + 1] * p[1] + G[3 * m + 2] * p[2]);
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
  }
  boost_inv(Y, e, p);
  const T rho = e;
  T mus = p[0] / e;
  mus = mus > T(1) ? T(1) : (mus < T(-1) ? T(-1) : mus);
  T phs = atan2_t(p[2], p[1]);
  if (phs < T(0)) phs += T(2 * kPi);
  // energy: eps* = rho eps_i, bracket eps_{i+m} <= eps* < eps_{i+m+1}
  // (t = rho / R^m formed as exp(log rho - m log R): one exponential in
  // place of a general power)
  const T lrho = log_t(rho);
  int m = (int)floor_t(lrho * K.rlR);
  T t = exp_t(lrho - (T)m * K.lR);
  T we = (t - T(1)) * K.rRm1;
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
    // the last node at or below mu* (a linear walk: measured faster than a
    // bisection on 8 nodes)
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
    T u = phs * (T(nph) * T(1.0 / (2 * kPi))) - T(0.5);
    T kf = floor_t(u);
    wp = u - kf;
    kL = ((int)kf) % nph;
    if (kL < 0) kL += nph;
  }
  w.wmu = wm; w.wph = wp; w.we = we;
  w.jL = (short)jL; w.kL = (short)kL; w.m = (short)m; w.pad = 0;
}

template <typename T>
__device__ __forceinline__ void chain_weights(const Tables& tb, const T* s_mu, const T* n0, const T* n1, const T* n2,
                                              const Loc<T>& X, const Loc<T>& Y, const T* G, int gT, int axis, int ang,
                                              const EBr<T>& K, Wt<T>& w) {
  const T n[3] = {n0[ang], n1[ang], n2[ang]};
  chain_weights_dir(tb, s_mu, n, X, Y, G, gT, axis, K, w);
}

// ---------------------------------------------------------------------------
// Double-float (pairs of float32) for exact-enough sums on the FP32 pipes
// ---------------------------------------------------------------------------
struct ff {
  float hi, lo;
};
// error-free sum of two floats (Knuth's TwoSum)
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return ff{s, e};
}
__device__ __forceinline__ ff ff_add(ff a, float b) {
  ff s = two_sum(a.hi, b);
  float lo = s.lo + a.lo;
  float hi = s.hi + lo;
  return ff{hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  float lo = s.lo + (a.lo + b.lo);
  float hi = s.hi + lo;
  return ff{hi, lo - (hi - s.hi)};
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_shfl_down(ff a, int o) {
  return ff{__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}
__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
  return ff{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}
// |a| >= |b| (Dekker's Fast2Sum)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = a + b;
  return ff{s, b - (s - a)};
}
// error-free product with a fused multiply-add
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  float lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return fast_two_sum(p.hi, lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
// 1/d by one Newton step from the float reciprocal: x + x e, e = 1 - d x
// (__frcp_rn: the correctly rounded reciprocal, the value of 1.0f / d.hi).
// |e| <= 2^-24, and 1 - d.hi x has at most 24 significant bits, so the inner
// fused multiply-add forms it exactly; the outer one adds -d.lo x with one
// rounding (2^-48 absolute).  The result has about 46 correct bits.
__device__ __forceinline__ ff ff_recip(ff d) {
  const float x = __frcp_rn(d.hi);
  const float e = fmaf(-d.lo, x, fmaf(-d.hi, x, 1.0f));
  return fast_two_sum(x, x * e);
}
__device__ __forceinline__ ff ff_from_d(double v) {
  float hi = (float)v;
  return ff{hi, (float)(v - (double)hi)};
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, 1D) into shared memory with an mbarrier.
// Every wait is bounded: on expiry the kernel raises st.flag[1].
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order earlier generic-proxy accesses of shared memory before later
// async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long kWaitLimit = 1L << 22;
// bounded wait for phase `parity`; returns false (and flags) on expiry
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* flag) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  flag[1] = 1;
  return false;
}

// ---------------------------------------------------------------------------
// The remap T applied as two gathers (Sec. 3.2, trilinear weights factorised
// into an energy part and an angular part):
//   energy pass:  E[t][b] = sum_i we(t | i, b) src[i][b]   (per source angle b:
//                 source group i goes to groups clamp(i+m_b) and clamp(i+m_b+1))
//   angular pass: D[t][b'] = sum_b wa(b' | b) E[t][b]      (per destination angle
//                 b': the source angles whose bracket contains b')
// The angular lists are built once per remap and serve every group and
// species; they are sorted by source angle so the summation order (and the
// result) is deterministic.
// ---------------------------------------------------------------------------
// Angular-list entries in two arrays: the weight (wmu * wphi) and the source
// angle, 6 bytes an entry in float32 (10 in float64); a remap's list starts
// at an offset of both (operator+)
template <typename T>
struct AList {
  T* w;
  short* b;
  __device__ __forceinline__ AList operator+(int o) const { return AList{w + o, b + o}; }
};
// Entry e of a remap's lists is stored at alist_at(e): one word of padding
// after every 32 entries.  The lanes of a warp read their lists about four
// entries apart, so without it lanes eight apart would hit one bank.
__host__ __device__ __forceinline__ int alist_at(int e) { return e + (e >> 5); }
// entries of one remap's block: 4 na entries (four targets per source angle)
// with their padding
__host__ __device__ __forceinline__ int alist_block(int na) { return alist_at(4 * na) + 1; }

// the angular targets of one source angle in four fixed slots (mu bracket
// lower/upper x Phi bracket lower/upper); a slot whose weight is zero, or
// that repeats another slot's target on a one-node axis (its weight merged
// there), is absent: tgt = -1
template <typename T>
__device__ __forceinline__ void ang_targets4(const Wt<T>& W, int nmu, int nph, int* tgt, T* wa) {
  const int jL = W.jL, kL = W.kL;
  const int jR = nmu >= 2 ? jL + 1 : jL;
  const int kR = nph >= 2 ? (kL + 1) % nph : kL;
  const T mj0 = T(1) - W.wmu, mj1 = W.wmu;
  const T mk0 = T(1) - W.wph, mk1 = W.wph;
  wa[0] = mj0 * mk0; wa[1] = mj0 * mk1; wa[2] = mj1 * mk0; wa[3] = mj1 * mk1;
  tgt[0] = jL * nph + kL; tgt[1] = jL * nph + kR; tgt[2] = jR * nph + kL; tgt[3] = jR * nph + kR;
  if (kR == kL) { wa[0] += wa[1]; wa[1] = T(0); wa[2] += wa[3]; wa[3] = T(0); }
  if (jR == jL) { wa[0] += wa[2]; wa[2] = T(0); wa[1] += wa[3]; wa[3] = T(0); }
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (wa[k] == T(0)) tgt[k] = -1;   // adds nothing: keep the lists short
}

// Build the angular lists of the remaps whose bit is set in `mask`, each
// destination's list sorted by source angle.  Every (remap, source) thread
// sets its bit in a per-destination bitmask of sources (atomicOr: the result
// does not depend on the order), the offsets are a scan of the masks' bit
// counts, and an entry's place in its list is the number of lower sources in
// the mask: no sorting pass, and all threads take part.
// off: [nr][na+1], msk: [nr][na][ceil(na/32)] scratch, ent: [nr][alist_block(na)]
// (entry e of a remap's lists at alist_at(e)).
// Whole block (synchronises at the end).
template <typename T>
__device__ void build_alists(const Wt<T>* W, int nr, unsigned mask, int na, int nmu, int nph, short* off,
                             unsigned* msk, AList<T> ent) {
  const int tid = threadIdx.x, nt = (int)blockDim.x;
  const int nwd = (na + 31) >> 5;
  for (int q = tid; q < nr * na * nwd; q += nt) msk[q] = 0u;
  __syncthreads();
  for (int q = tid; q < nr * na; q += nt) {
    const int r = q / na, b = q % na;
    if (!((mask >> r) & 1u)) continue;
    int tgt[4];
    T wa[4];
    ang_targets4(W[q], nmu, nph, tgt, wa);
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (tgt[k] >= 0) atomicOr(&msk[(r * na + tgt[k]) * nwd + (b >> 5)], 1u << (b & 31));
  }
  __syncthreads();
  {
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < nr; r += (nt >> 5)) {
      if (!((mask >> r) & 1u)) continue;
      const int per = (na + 31) / 32;
      const int k0 = min(lane * per, na), k1 = min(k0 + per, na);
      int loc = 0;
      for (int k = k0; k < k1; ++k)
        for (int w = 0; w < nwd; ++w) loc += __popc(msk[(r * na + k) * nwd + w]);
      int incl = loc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      int run = incl - loc;
      for (int k = k0; k < k1; ++k) {
        off[r * (na + 1) + k] = (short)run;
        for (int w = 0; w < nwd; ++w) run += __popc(msk[(r * na + k) * nwd + w]);
      }
      if (lane == 31) off[r * (na + 1) + na] = (short)incl;
    }
  }
  __syncthreads();
  for (int q = tid; q < nr * na; q += nt) {
    const int r = q / na, b = q % na;
    if (!((mask >> r) & 1u)) continue;
    int tgt[4];
    T wa[4];
    ang_targets4(W[q], nmu, nph, tgt, wa);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (tgt[k] < 0) continue;
      const unsigned* mt = msk + (r * na + tgt[k]) * nwd;
      int pos = off[r * (na + 1) + tgt[k]];
      for (int w = 0; w < (b >> 5); ++w) pos += __popc(mt[w]);
      pos += __popc(mt[b >> 5] & ((1u << (b & 31)) - 1u));
      ent.w[r * alist_block(na) + alist_at(pos)] = wa[k];
      ent.b[r * alist_block(na) + alist_at(pos)] = (short)b;
    }
  }
  __syncthreads();
}

// Layout of the energy pass's output (the angular pass's input): a thread
// of chunk gc handles rows t = gc + k nch (k = 0, 1, ...) of its column;
// those rows of column b are contiguous, E[(gc na + b) rpt + k], so that the
// angular pass reads a block of rows of one source angle at immediate
// offsets from one address.  rpt: the rows of a chunk rounded up to whole
// blocks of rb, and to an odd count (consecutive columns then fall in
// different shared-memory banks).
__host__ __device__ __forceinline__ int chunk_nch(int na, int nt) { return nt / na > 0 ? nt / na : 1; }
__host__ __device__ __forceinline__ int chunk_rpt(int ne, int na, int nt, int rb) {
  const int nch = chunk_nch(na, nt);
  const int rows = (ne + nch - 1) / nch;
  int r = (rows + rb - 1) / rb * rb;
  return (r & 1) ? r : r + 1;
}
// elements of one energy-pass output buffer (at least ne na, a multiple of 4)
__host__ __device__ __forceinline__ size_t chunk_elems(int ne, int na, int nt, int rb) {
  size_t n = (size_t)chunk_nch(na, nt) * na * chunk_rpt(ne, na, nt, rb);
  if (n < (size_t)ne * na) n = (size_t)ne * na;
  return (n + 3) & ~size_t(3);
}

// Energy pass for column b (source angle b, shift m, upper weight we) in
// "y-form" (content per unit dGamma): source group i goes to groups
// clamp(i+m) (weight 1-we) and clamp(i+m+1) (we), and its content per unit
// dGamma is rescaled by dGamma_i / dGamma_t = R^(3(i-t)) (p3c[k] = R^(3k)):
//   E[t] = c * sum_i w(t|i) R^(3(i-t)) src[i].
// the first and last group's rows (clamped targets); the flux kernel calls
// them through energy_edge, not inlined, which keeps its hot loop small (its
// instruction fetch stalls otherwise; the same rows, the same sums)
template <typename T, typename A>
__device__ __forceinline__ A energy_edge_inl(int t, int ne, int na, int b, int m, A wl, A wr, const T* src,
                                             const T* p3c) {
  A acc = A(0);
  int lo = (t == 0) ? 0 : t - m;
  int hi = (t == ne - 1) ? ne - 1 : t - m;
  lo = max(lo, 0); hi = min(hi, ne - 1);
  for (int i = lo; i <= hi; ++i) acc += wl * (A)p3c[i - t] * (A)src[i * na + b];
  lo = (t == 0) ? 0 : t - m - 1;
  hi = (t == ne - 1) ? ne - 1 : t - m - 1;
  lo = max(lo, 0); hi = min(hi, ne - 1);
  for (int i = lo; i <= hi; ++i) acc += wr * (A)p3c[i - t] * (A)src[i * na + b];
  return acc;
}

template <typename T, typename A>
__device__ __noinline__ A energy_edge(int t, int ne, int na, int b, int m, A wl, A wr, const T* src, const T* p3c) {
  return energy_edge_inl<T, A>(t, ne, na, b, m, wl, wr, src, p3c);
}

// products and sums that the compiler may not fuse: code inlined into
// several kernels (the fused and the split flux forms) must round the same
// way in each of them
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// The first (top = false) and last (top = true) group's rows for shifts of
// less than one group (m = 0 or -1) and at least two groups: the clamped
// taps of energy_edge_inl in closed form, the same terms in the same order
// (no call, no loop: the common case of every remap)
template <typename T, typename A>
__device__ __forceinline__ A energy_edge_fast(bool top, int ne, int na, int b, int m, A wl, A wr, const T* src,
                                              const T* p3c) {
  if (!top) {
    const A s0 = (A)src[b];
    A acc = mul_rn(mul_rn(wl, (A)p3c[0]), s0);
    if (m == -1) {
      acc = add_rn(acc, mul_rn(mul_rn(wl, (A)p3c[1]), (A)src[na + b]));
      acc = add_rn(acc, mul_rn(mul_rn(wr, (A)p3c[0]), s0));
    }
    return acc;
  }
  const int t = ne - 1;
  const A st = (A)src[t * na + b];
  if (m == -1) return mul_rn(mul_rn(wr, (A)p3c[0]), st);
  A acc = mul_rn(mul_rn(wl, (A)p3c[0]), st);
  acc = add_rn(acc, mul_rn(mul_rn(wr, (A)p3c[-1]), (A)src[(t - 1) * na + b]));
  acc = add_rn(acc, mul_rn(mul_rn(wr, (A)p3c[0]), st));
  return acc;
}

// (src: rows [group][angle]; E: the chunk layout above, rpt its row count)
template <typename T, typename A, bool kEdgeCall = false>
__device__ __forceinline__ void energy_column(int gc, int nch, int ne, int na, int b, int m, T we, const T* src, T* E,
                                              int rpt, T c, const T* p3c) {
  T* Ec = E + (size_t)(gc * na + b) * rpt;   // row t = gc + k nch at Ec[k]
  const A wl = (A)c * (A(1) - (A)we), wr = (A)c * (A)we;
  const bool small = m > -ne && m < ne;   // interior sources exist only then
  const A wli = small ? wl * (A)p3c[-m] : A(0);
  const A wri = (m >= -ne && m < ne - 1) ? wr * (A)p3c[-m - 1] : A(0);
  if (__all_sync(__activemask(), m == 0 || m == -1)) {
    // shifts of less than one group (the usual case): both taps of every
    // interior row lie in range, so the rows need no bounds checks; the
    // edge rows as below.  Same operations in the same order.
    int t = gc;
    T* Ek = Ec;
    if (t == 0) {
      *Ek++ = (T)(ne >= 2 ? energy_edge_fast<T, A>(false, ne, na, b, m, wl, wr, src, p3c)
                  : kEdgeCall ? energy_edge<T, A>(0, ne, na, b, m, wl, wr, src, p3c)
                              : energy_edge_inl<T, A>(0, ne, na, b, m, wl, wr, src, p3c));
      t += nch;
    }
    const T* sL = src + (t - m) * na + b;   // tap t - m; the other tap is one row lower
    for (; t < ne - 1; t += nch, sL += nch * na) {
      A acc = A(0);
      acc += wli * (A)sL[0];
      acc += wri * (A)sL[-na];
      *Ek++ = (T)acc;
    }
    if (t == ne - 1)   // here t >= 1, so at least two groups
      *Ek = (T)energy_edge_fast<T, A>(true, ne, na, b, m, wl, wr, src, p3c);
    return;
  }
  for (int t = gc, k = 0; t < ne; t += nch, ++k) {
    A acc = A(0);
    if (t > 0 && t < ne - 1) {
      int iL = t - m, iR = t - m - 1;
      if (iL >= 0 && iL < ne) acc += wli * (A)src[iL * na + b];
      if (iR >= 0 && iR < ne) acc += wri * (A)src[iR * na + b];
    } else if (kEdgeCall) {
      acc = energy_edge<T, A>(t, ne, na, b, m, wl, wr, src, p3c);
    } else {
      acc = energy_edge_inl<T, A>(t, ne, na, b, m, wl, wr, src, p3c);
    }
    Ec[k] = (T)acc;
  }
}

// energy_column for one remap, not inlined (the rare path of energy_cells)
template <typename T, typename A>
__device__ __noinline__ void energy_column_call(int gc, int nch, int ne, int na, int b, int m, T we, const T* src,
                                                T* E, int rpt, T c, const T* p3c) {
  energy_column<T, A, true>(gc, nch, ne, na, b, m, we, src, E, rpt, c, p3c);
}

// The energy pass of up to NC remaps of one source column together (the same
// source angle b; remap q with its shift m[q], weight we[q], density factor
// c[q], source rows src[q] and output E[q]; bit q of act: remap q present,
// the same for the whole block).  Where the shifts of every present remap in
// the warp are below one group, the rows are walked once for all of them
// (the same operations per row as energy_column's); otherwise each remap
// takes energy_column.
template <int NC, typename T, typename A>
__device__ __forceinline__ void energy_cells(int gc, int nch, int ne, int na, int b, unsigned act, const int* m,
                                             const T* we, const T* c, const T* const* src, T* const* E, int rpt,
                                             const T* p3c) {
  bool small = true;
#pragma unroll
  for (int q = 0; q < NC; ++q)
    if ((act >> q) & 1u) small = small && (m[q] == 0 || m[q] == -1);
  if (!__all_sync(__activemask(), small) || ne < 2) {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if ((act >> q) & 1u) energy_column_call<T, A>(gc, nch, ne, na, b, m[q], we[q], src[q], E[q], rpt, c[q], p3c);
    return;
  }
  A wl[NC], wr[NC], wli[NC], wri[NC];
  T* Ec[NC];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    wl[q] = (A)c[q] * (A(1) - (A)we[q]);
    wr[q] = (A)c[q] * (A)we[q];
    wli[q] = wl[q] * (A)p3c[-m[q]];
    wri[q] = wr[q] * (A)p3c[-m[q] - 1];
    Ec[q] = E[q] + (size_t)(gc * na + b) * rpt;   // row t = gc + k nch at Ec[q][k]
  }
  int t = gc, k = 0;
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if ((act >> q) & 1u) Ec[q][0] = (T)energy_edge_fast<T, A>(false, ne, na, b, m[q], wl[q], wr[q], src[q], p3c);
    t += nch;
    k = 1;
  }
  for (; t < ne - 1; t += nch, ++k) {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if ((act >> q) & 1u) {
        const T* sL = src[q] + (t - m[q]) * na + b;   // tap t - m; the other tap one row lower
        A acc = A(0);
        acc += wli[q] * (A)sL[0];
        acc += wri[q] * (A)sL[-na];
        Ec[q][k] = (T)acc;
      }
  }
  if (t == ne - 1) {
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if ((act >> q) & 1u) Ec[q][k] = (T)energy_edge_fast<T, A>(true, ne, na, b, m[q], wl[q], wr[q], src[q], p3c);
  }
}

// Angular pass for destination angle bp over the rows of this thread:
// out(t) = sum_e w_e E[t][b_e], the entries summed in list order.  Rows are
// taken RB at a time and each list entry is read once for the RB rows, whose
// values of its source angle are contiguous in the chunk layout (Eb: the
// block's first row of source angle 0; a source's rows at Eb + b rpt + j).
// The lanes of a warp walk the entries together up to the longest list among
// them (a lane with a shorter list skips the rest), so lists of uneven length
// do not split the warp into separate passes.  Rows past the last group
// (padding of the block) are read but never stored.
template <int RB, typename T, typename A, typename Out>
__device__ __forceinline__ void angular_block(int t0, int nch, int ne, const T* Eb, int rpt, int e0, int n, int nmax,
                                              AList<T> ent, Out out) {
  A acc[RB];
#pragma unroll
  for (int j = 0; j < RB; ++j) acc[j] = A(0);
#pragma unroll 2
  for (int k = 0; k < nmax; ++k) {
    if (k < n) {
      const int e = alist_at(e0 + k);
      const A w = (A)ent.w[e];
      const T* eb = Eb + ent.b[e] * rpt;
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[j] += w * (A)eb[j];
    }
  }
#pragma unroll
  for (int j = 0; j < RB; ++j) {
    const int t = t0 + j * nch;
    if (t < ne) out(t, acc[j]);
  }
}

// RB rows per walk of the lists (the kernels pick it from the rows a thread
// holds); E in the chunk layout with rpt rows per column
template <typename T, typename A, int RB, typename Out>
__device__ __forceinline__ void angular_rows(int gc, int nch, int ne, int na, int rpt, int e0, int e1, AList<T> ent,
                                             const T* E, Out out) {
  const int n = e1 - e0;
  const int nmax = __reduce_max_sync(__activemask(), n);
  const T* Eg = E + (size_t)gc * na * rpt;
  for (int t0 = gc, blk = 0; t0 < ne; t0 += RB * nch, ++blk)
    angular_block<RB, T, A>(t0, nch, ne, Eg + blk * RB, rpt, e0, n, nmax, ent, out);
}

// Pole nodes of a Gauss-Lobatto mu grid (mu = -1 and +1): the n_ph cells of
// such a node are one direction, so content the remap moves into the node is
// spread evenly over them.  The angular pass deposits with linear Phi
// weights; replacing each pole node's cells by their mean, row by row, gives
// the even spread (the node's total is unchanged) and does not depend on Phi*,
// which is ill-conditioned next to the pole.  X: [nrows][na]; whole block,
// no barrier inside (the caller synchronises before and after).
template <typename T>
__device__ __forceinline__ void pole_mean(T* X, int nrows, int na, int nmu, int nph) {
  for (int q = threadIdx.x; q < 2 * nrows; q += blockDim.x) {
    T* c = X + (size_t)(q >> 1) * na + ((q & 1) ? (nmu - 1) * nph : 0);
    T sum = T(0);
    for (int k = 0; k < nph; ++k) sum += c[k];
    sum = sum / T(nph);
    for (int k = 0; k < nph; ++k) c[k] = sum;
  }
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
  F.bc = 0;
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
      if (edge == 0 || (edge == tb.n_th && !tb.th_open)) return false;
      F.area = tb.area_t[edge * nr + a];
      F.own = fidx == 2 ? 2 : 1;
      if (edge == tb.n_th) { F.type = F_OUTFLOW_P; F.bc = 1; }   // the open face at theta_max
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

__device__ __forceinline__ double pow6(double x) {
  double x2 = x * x;
  return x2 * x2 * x2;
}

// Face constants in the arithmetic type (staged once per face).
template <typename T>
struct FaceT {
  T dt;                     // the face's step (the step of its finer side under local time stepping)
  T xs, dx, area, al, cf, c6;
  T sP, sQ;                 // xs - x1, xs - x2
  T rdx, rdl0, rdl1, rdl2;  // reciprocals of dx and the stencil spacings
  T c6k[4];                 // phi^6 of the stencil cells
};

constexpr int kFaces = 5;
constexpr int kSurKindsAll = 1 + 6 * kFaces;   // remap kinds of a zone (learned remap table)

// dN accumulator type: float64 for the FP64 path; float for the mixed path,
// whose per-zone content totals are tracked exactly (double-float) and
// restored before the collision solve.
template <typename T>
struct DNT;
template <>
struct DNT<double> { using type = double; };
template <>
struct DNT<float> { using type = float; };

// Shared-memory carve-up of the flux kernel.  mode 0: fused faces +
// collision of one zone; mode 1: the face pass (no dN); mode 2: the zone
// pass (no stencil buffers or lists).
template <typename T>
struct FluxSmem {
  typename DNT<T>::type* dN;  // [ns][ne][nang]
  double* zu0;     // [nang] own zone u^0
  double* ztau;    // [nang] alpha dt / u^0
  double* zcn;     // [nang] 1/(phi^6 dV u^0 dOmega)
  ff* zt_f;        // [nang] double-float copies of tau, zcn, dOmega (mixed collision)
  ff* zc_f;
  ff* zd_f;
  float* zq_f;     // [nang] phi^6 u^0 dOmega / dt
  double* zrow;    // [ns][ne][5] collision moment partials
  ff* rowk;        // [ns][ne][4] ka, ks, ka + ks, ka f_eq of each row (mixed solve)
  double* wr_r;    // [warps][nang] f* of the warp's collision row   (aliases buf)
  double* wr_i;    // [warps][nang] 1/D per warp row                 (aliases buf)
  double* red;     // [kMaxWarps * 2]
  double* zsc;     // [8] the zone's float64 scalars of the collision (formed once)
  double* tally;   // [ns][2] outflow N, E of this zone
  double* corr;    // [ns] exact-total correction of dN (mixed)
  ff* corr_f;      // [ns] the same as a double-float
  int* corr_at;    // [ns]
  ff* dtot;        // [ns] exact total of the deposits (mixed)
  ff* redf;        // [kMaxWarps]
  ff* redfS;       // [ns][kMaxWarps] per-species warp sums (zone pass)
  float* rkeyS;    // [ns][kMaxWarps]
  int* ridxS;      // [ns][kMaxWarps]
  float* rkey;     // [kMaxWarps]
  int* ridx;       // [kMaxWarps]
  unsigned long long* bar;  // mbarrier of the stencil copies
  T* buf;          // [8][ne][nang]: 4 stencil/g buffers, 4 work buffers
  Wt<T>* W;        // [6][nang]   (aliases the work buffers)
  unsigned* msk;   // [6][nang][ceil(nang/32)] (aliases the work buffers)
  AList<T> ent;    // [6][4 nang]
  short* off;      // [6][nang + 1]
  T* n0; T* n1; T* n2;  // [nang] direction components
  T* dOm;          // [nang]
  T* dGam;         // [ne]
  T* rdGam;        // [ne] 1/dGamma
  T* epsS;         // [ne] group centres
  T* mu;           // [nmu]
  T* u0s;          // [nang] face
  T* vns;          // [nang]
  T* cs;           // [nang] 1/(phi_s^6 u0_s dOmega)
  T* taus;         // [nang] (dt/2) alpha_s / u0_s
  T* vdx;          // [nang] (dt/2) v_s / dx
  T* rowJ;         // [ne]
  T* kaS; T* ksS; T* feS; T* wP; T* wQ;  // [ne]
  FaceDesc* F;     // [kFaces]
  FaceT<T>* FT;    // [kFaces]
  Loc<T>* L;       // [kFaces][5] boosts of the stencil cells (0..3) and the face (4)
  T* Gs;           // [kFaces][4][9] rotations stencil cell -> face in T
  T* p3;           // [2 ne + 3] R^(3k)
};

// rows per angular-list walk (RB) of a kernel of nt threads, unless the
// launch picks another (face_rb)
__host__ __device__ constexpr int default_rb(int nt) { return nt >= 512 ? 2 : 4; }

template <typename T>
__host__ __device__ size_t flux_smem_layout(int ns, int ne, int nang, int nmu, int nw, int mode, int rb, FluxSmem<T>* s,
                                           unsigned char* base) {
  size_t o = 0;
  const int nbin = ne * nang;
#define BT_TAKE(ptr, type, count)                              \
  do {                                                         \
    o = (o + 15) & ~size_t(15);                                \
    if (s) s->ptr = reinterpret_cast<type*>(base + o);         \
    o += sizeof(type) * (size_t)(count);                       \
  } while (0)
  BT_TAKE(bar, unsigned long long, 2);
  BT_TAKE(dN, typename DNT<T>::type, mode == 0 ? (size_t)ns * nbin : 0);   // fused kernel only
  const int nz_ang = mode == 1 ? 0 : nang;   // the collision's arrays: not in the face pass
  BT_TAKE(zu0, double, nz_ang);
  BT_TAKE(ztau, double, nz_ang);
  BT_TAKE(zcn, double, nz_ang);
  BT_TAKE(zt_f, ff, nz_ang);
  BT_TAKE(zc_f, ff, nz_ang);
  BT_TAKE(zd_f, ff, nz_ang);
  BT_TAKE(zq_f, float, nz_ang);
  BT_TAKE(zrow, double, mode == 1 ? 0 : (size_t)ns * ne * 5);
  BT_TAKE(rowk, ff, mode == 1 ? 0 : (size_t)ns * ne * 4);
  BT_TAKE(red, double, kMaxWarps * 2);
  BT_TAKE(zsc, double, mode == 1 ? 0 : 8);
  BT_TAKE(tally, double, ns * 2);
  BT_TAKE(corr, double, mode == 1 ? 0 : ns);   // the corrections: not in the face pass
  BT_TAKE(corr_f, ff, mode == 1 ? 0 : ns);
  BT_TAKE(corr_at, int, mode == 1 ? 0 : ns);
  BT_TAKE(dtot, ff, ns);
  BT_TAKE(redf, ff, kMaxWarps);
  BT_TAKE(redfS, ff, mode == 2 ? (size_t)ns * kMaxWarps : 0);
  BT_TAKE(rkeyS, float, mode == 2 ? (size_t)ns * kMaxWarps : 0);
  BT_TAKE(ridxS, int, mode == 2 ? (size_t)ns * kMaxWarps : 0);
  BT_TAKE(rkey, float, kMaxWarps);
  BT_TAKE(ridx, int, kMaxWarps);
  {
    // buf = 4 stencil buffers followed by 4 work buffers.  The remap weights
    // and list bitmasks live only until the lists are built, when the work
    // buffers are idle; the collision scratch only after the last face.
    size_t o_b = (o + 15) & ~size_t(15);
    size_t stencil = sizeof(T) * (size_t)4 * nbin;
    size_t o_work = o_b + stencil;
    size_t o_c = (o_work + sizeof(Wt<T>) * (size_t)6 * nang + 15) & ~size_t(15);
    // the work buffers hold the energy passes' outputs in the chunk layout
    size_t need_work = sizeof(T) * (size_t)4 * chunk_elems(ne, nang, nw * 32, rb);
    size_t need_wc = o_c + sizeof(unsigned) * (size_t)6 * nang * ((nang + 31) / 32) - o_work;
    size_t need_col = sizeof(double) * (size_t)2 * nw * nang;
    size_t tot = stencil + (need_work > need_wc ? need_work : need_wc);
    if (mode == 2) tot = 0;   // the zone pass stages no stencils
    if (need_col > tot) tot = need_col;
    if (s) {
      s->buf = reinterpret_cast<T*>(base + o_b);
      s->W = reinterpret_cast<Wt<T>*>(base + o_work);
      s->msk = reinterpret_cast<unsigned*>(base + o_c);
      s->wr_r = reinterpret_cast<double*>(base + o_b);
      s->wr_i = reinterpret_cast<double*>(base + o_b) + (size_t)nw * nang;
    }
    o = o_b + tot;
  }
  BT_TAKE(ent.w, T, mode == 2 ? 0 : 6 * alist_block(nang));
  BT_TAKE(ent.b, short, mode == 2 ? 0 : 6 * alist_block(nang));
  BT_TAKE(off, short, mode == 2 ? 0 : 6 * (nang + 1));
  BT_TAKE(n0, T, nang);
  BT_TAKE(n1, T, nang);
  BT_TAKE(n2, T, nang);
  BT_TAKE(dOm, T, nang);
  BT_TAKE(dGam, T, ne);
  BT_TAKE(rdGam, T, ne);
  BT_TAKE(epsS, T, ne);
  BT_TAKE(mu, T, nmu);
  BT_TAKE(u0s, T, nang);
  BT_TAKE(vns, T, nang);
  BT_TAKE(cs, T, nang);
  BT_TAKE(taus, T, nang);
  BT_TAKE(vdx, T, nang);
  BT_TAKE(rowJ, T, ne);
  BT_TAKE(kaS, T, mode == 2 ? 0 : (size_t)ns * ne);
  BT_TAKE(ksS, T, mode == 2 ? 0 : (size_t)ns * ne);
  BT_TAKE(feS, T, mode == 2 ? 0 : (size_t)ns * ne);
  BT_TAKE(wP, T, mode == 2 ? 0 : (size_t)ns * ne);
  BT_TAKE(wQ, T, mode == 2 ? 0 : (size_t)ns * ne);
  BT_TAKE(F, FaceDesc, kFaces);
  BT_TAKE(FT, FaceT<T>, kFaces);
  BT_TAKE(L, Loc<T>, kFaces * 5);
  BT_TAKE(Gs, T, kFaces * 36);
  BT_TAKE(p3, T, 2 * ne + 3);
#undef BT_TAKE
  return (o + 15) & ~size_t(15);
}

template <typename T>
__device__ __forceinline__ T mc_limiter(T a, T b) {
  // symmetric in a and b, bit for bit; no branch (selects)
  const T s = a > T(0) ? T(1) : T(-1);
  const T x = fabs(T(2) * a), y = fabs(T(2) * b), z = T(0.5) * fabs(a + b);
  T m = x < y ? x : y;
  m = m < z ? m : z;
  return a * b <= T(0) ? T(0) : s * m;
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
  for (int i = 0; i < ((int)blockDim.x >> 5); ++i) { s0 += red[2 * i]; s1 += red[2 * i + 1]; }
  __syncthreads();
  out1 = s1;
  return s0;
}

// deterministic block sum of double-floats (result in every thread)
__device__ __forceinline__ ff block_sum_ff(ff v, ff* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_down(v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  ff t = red[0];
  for (int i = 1; i < ((int)blockDim.x >> 5); ++i) t = ff_add(t, red[i]);
  __syncthreads();
  return t;
}

// block argmax of key >= 0 (ties -> smallest index); result in every thread
__device__ __forceinline__ int block_argmax(float key, int idx, float* rk, int* ri) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float k2 = __shfl_down_sync(0xffffffffu, key, o);
    int i2 = __shfl_down_sync(0xffffffffu, idx, o);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { rk[w] = key; ri[w] = idx; }
  __syncthreads();
  float bk = rk[0];
  int bi = ri[0];
  for (int i = 1; i < ((int)blockDim.x >> 5); ++i)
    if (rk[i] > bk || (rk[i] == bk && ri[i] < bi)) { bk = rk[i]; bi = ri[i]; }
  __syncthreads();
  return bi;
}
template <typename T>
struct StoreG {   // g = D / (phi_s^6 u0_s dOmega) in the face frame (D per unit dGamma)
  T* dst; T cs; int na, b;
  __device__ void operator()(int t, T acc) const { dst[t * na + b] = acc * cs; }
};
template <typename T>
struct StoreT {
  T* dst; int na, b;
  __device__ void operator()(int t, T acc) const { dst[t * na + b] = acc; }
};

// ---------------------------------------------------------------------------
// Fused face fluxes + collision of one zone (Sec. 3.3, 3.5, 3.4)
// ---------------------------------------------------------------------------
// Split form: a face pass computes every face once (CTA per zone over the
// faces it owns) and writes both neighbours' deposits; a zone pass gathers a
// zone's deposits in the fused kernel's order and solves the collision.
// Deposit rows live at slot 2 axis + (zone is the face's P side) of the
// receiving zone: dep[(zone * 6 + slot) * n_s + s][group][angle].
struct DepRec {
  ff sum;           // exact total of the deposit row (mixed path)
  double tn, te;    // outflow number and energy at infinity through the face
};

template <typename T>
struct StoreDep {   // dep = sign * T[F], or dep += sign * T[F] (a step that began earlier)
  T* dst; int na, b; T sign; bool add;
  __device__ void operator()(int t, T acc) const {
    T* d = dst + t * na + b;
    *d = add ? *d + sign * acc : sign * acc;
  }
};

// a zone's faces owned by it in the face pass (each face has one owner)
__device__ __forceinline__ bool face_owned(const Tables& tb, int a, int fidx) {
  if (fidx == 0) return a == 0;
  if (fidx == 2) return tb.periodic_th != 0;
  return true;
}

// existence of a zone's face fidx, as make_face decides it
__device__ __forceinline__ bool face_exists(const Tables& tb, int a, int b, int fidx) {
  const int nr = tb.n_r;
  if (fidx == 0 || fidx == 1) return tb.area_r[b * (nr + 1) + (fidx == 0 ? a : a + 1)] != 0.0;
  if (tb.slab) return false;
  if (fidx == 2 || fidx == 3) {
    if (tb.periodic_th) return fidx == 2 && tb.area_t[a] != 0.0;
    const int edge = fidx == 2 ? b : b + 1;
    if (edge == 0 || (edge == tb.n_th && !tb.th_open)) return false;
    return tb.area_t[edge * nr + a] != 0.0;
  }
  return tb.area_p[b * nr + a] != 0.0;
}

// The zone pass's exact deposit totals and outflow tallies from the face
// pass's records: lane s of the calling warp sums species s's records (faces
// in order, Q side then P side) in registers, the species in parallel.  Not
// inlined: inlined into the zone pass it raised that kernel's registers from
// 48 to 92.
__device__ __noinline__ void zone_records(const Tables& tb, const DepRec* rec, int zone, int a, int b, int nface,
                                          int NS, bool mixed, ff* dtot, double* tally) {
  const int lane = threadIdx.x & 31;
  for (int s = lane; s < NS; s += 32) {
    ff dt = dtot[s];
    double t0 = tally[2 * s], t1 = tally[2 * s + 1];
    for (int fidx = 0; fidx < nface; ++fidx) {
      if (!face_exists(tb, a, b, fidx)) continue;
      const int axis = fidx < 2 ? 0 : (fidx < 4 ? 1 : 2);
      const bool isP = fidx == 1 || fidx == 3 || fidx == 4 || (fidx == 2 && tb.periodic_th);
      const bool isQ = fidx == 0 || fidx == 4 || (fidx == 2);
      const DepRec* rP = isP ? rec + ((size_t)zone * 6 + 2 * axis + 1) * NS + s : nullptr;
      const DepRec* rQ = isQ ? rec + ((size_t)zone * 6 + 2 * axis) * NS + s : nullptr;
      if (mixed) {
        if (rQ) dt = ff_add(dt, rQ->sum);
        if (rP) dt = ff_add(dt, rP->sum);
      }
      // an outflow face has one side; the other side's record holds 0
      const double tn = (rP ? rP->tn : 0.0) + (rQ ? rQ->tn : 0.0);
      const double te = (rP ? rP->te : 0.0) + (rQ ? rQ->te : 0.0);
      if (tn != 0.0 || te != 0.0) { t0 += tn; t1 += te; }
    }
    dtot[s] = dt;
    tally[2 * s] = t0;
    tally[2 * s + 1] = t1;
  }
}

template <typename T>
struct AddDN {   // dN += sign * T[F]
  typename DNT<T>::type* dn; int na, b; T sign;
  __device__ void operator()(int t, T acc) const { dn[t * na + b] += (typename DNT<T>::type)(sign * acc); }
};

// RB: rows per angular-list walk (angular_rows); the default is the one the
// fused kernel and the zone pass use
template <typename T, int NT, int MODE, int RB = default_rb(NT), int NEC = 0, int NAC = 0, int NMUC = 0, int NPHC = 0>
__device__ __forceinline__ void flux_body(const Tables& tb, const State& st, double dt, T* dep, DepRec* rec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using DN = typename DNT<T>::type;
  // paired loads in the zone pass's gather (registers allow them where the
  // grid is fixed at compile time)
  constexpr bool kPair = NEC > 0;
  FluxSmem<T> S;
  flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, NT / 32, MODE, RB, &S, smem_raw);
  const int zone = st.zlist ? st.zlist[blockIdx.x] : (int)blockIdx.x;
  const int a = zone % tb.n_r, b = zone / tb.n_r;
  // local time stepping: the zone pass takes the zone's own step
  const bool lts = st.lev != nullptr;
  if (lts && MODE == 2) dt = st.dt0 * (double)(1 << st.lev[zone]);
  const int NE = NEC ? NEC : tb.n_e, NA = NAC ? NAC : tb.n_ang, NS = tb.n_s;
  const int NPH = NPHC ? NPHC : tb.n_ph, NMU = NMUC ? NMUC : tb.n_mu;
  const int nbin = NE * NA;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nch = NT / NA > 0 ? NT / NA : 1;   // row chunks
  const int gb = tid % NA, gc = tid / NA;                   // this thread's angle, chunk
  const bool gact = tid < nch * NA;
  const T* fin = reinterpret_cast<const T*>(st.f);
  T* fout = reinterpret_cast<T*>(st.f_next);
  T* const SRC = S.buf;              // [4] stencil f rows (TMA), then g (face f values)
  T* const EB = S.buf + 4 * nbin;    // [4] work buffers of ebs elements
  const int ebs = (int)chunk_elems(NE, NA, NT, RB);
  const int rpt = chunk_rpt(NE, NA, NT, RB);   // rows per column in the chunk layout
  const unsigned rowbytes = (unsigned)(sizeof(T) * (size_t)nbin);
  const bool use_tma = (rowbytes % 16u) == 0u;
  unsigned tphase = 0;               // parity of the next mbarrier phase to wait for
  const T dtT = (T)dt;               // converted once

  if (MODE == 0)
    for (int q = tid; q < NS * nbin; q += NT) S.dN[q] = DN(0);
  // the zone's summed deposits [s][group][angle]: shared memory in the fused
  // kernel; in the zone pass, the zone's first deposit slot (set below)
  if constexpr (sizeof(T) == 4) {
    // the float32 tables (no per-CTA float64 conversions)
    for (int q = tid; q < NMU; q += NT) S.mu[q] = tb.f_mu[q];
    for (int q = tid; q < NA; q += NT) {
      S.n0[q] = tb.f_n0[q]; S.n1[q] = tb.f_n1[q]; S.n2[q] = tb.f_n2[q]; S.dOm[q] = tb.f_dOm[q];
    }
    for (int q = tid; q < NE; q += NT) { S.dGam[q] = tb.f_dGam[q]; S.rdGam[q] = tb.f_rdGam[q]; S.epsS[q] = tb.f_eps[q]; }
    for (int q = tid; q < 2 * NE + 3; q += NT) S.p3[q] = tb.f_p3[q];
  } else {
    for (int q = tid; q < NMU; q += NT) S.mu[q] = (T)tb.mu[q];
    for (int q = tid; q < NA; q += NT) {
      int j = q / NPH, k = q % NPH;
      S.n0[q] = (T)tb.mu[j];
      S.n1[q] = (T)(tb.smu[j] * tb.cph[k]);
      S.n2[q] = (T)(tb.smu[j] * tb.sph[k]);
      S.dOm[q] = (T)tb.dOm[q];
    }
    for (int q = tid; q < NE; q += NT) {
      S.dGam[q] = (T)tb.dGam[q];
      S.rdGam[q] = (T)(1.0 / tb.dGam[q]);
      S.epsS[q] = (T)tb.eps[q];
    }
    for (int q = tid; q < 2 * NE + 3; q += NT) S.p3[q] = (T)tb.p3[q];
  }
  for (int q = tid; q < NS * 2; q += NT) S.tally[q] = 0.0;
  for (int q = tid; q < NS; q += NT) S.dtot[q] = ff{0.0f, 0.0f};
  if (tid == 0) mbar_init(S.bar, 1);
  const int nface = tb.slab ? 2 : kFaces;
  if (MODE != 2 && tid < nface) {
    FaceDesc& Fd = S.F[tid];
    int lf = 0;   // local time stepping: the face's level (its finer side's)
    bool active = true;
    if ((MODE == 1 && !face_owned(tb, a, tid)) || !make_face(tb, st, a, b, tid, Fd)) {
      active = false;
    } else if (lts) {
      lf = Fd.z[1] >= 0 ? st.lev[Fd.z[1]] : st.lev[Fd.z[2]];
      if (Fd.z[1] >= 0 && Fd.z[2] >= 0) lf = min(lf, st.lev[Fd.z[2]]);
      active = (st.lts_k % (1 << lf)) == 0;   // evaluated when its finer side starts a step
      // a side whose own step began at an earlier substep adds to its row
      Fd.addP = Fd.z[1] >= 0 && (st.lts_k % (1 << st.lev[Fd.z[1]])) != 0;
      Fd.addQ = Fd.z[2] >= 0 && (st.lts_k % (1 << st.lev[Fd.z[2]])) != 0;
    } else {
      Fd.addP = Fd.addQ = 0;
    }
    if (!active) {
      Fd.type = -1;
    } else {
      FaceT<T>& ft = S.FT[tid];
      ft.dt = lts ? (T)(st.dt0 * (double)(1 << lf)) : dtT;
      ft.xs = (T)Fd.xs; ft.dx = (T)Fd.dx; ft.area = (T)Fd.area;
      ft.al = (T)Fd.al; ft.cf = (T)Fd.cf; ft.c6 = (T)pow6(Fd.cf);
      ft.sP = (T)(Fd.xs - Fd.x[1]); ft.sQ = (T)(Fd.xs - Fd.x[2]);
      ft.rdx = (T)(1.0 / Fd.dx);
      ft.rdl0 = Fd.z[0] >= 0 ? (T)(1.0 / (Fd.x[1] - Fd.x[0])) : T(0);
      ft.rdl1 = (T)(1.0 / (Fd.x[2] - Fd.x[1]));
      ft.rdl2 = Fd.z[3] >= 0 ? (T)(1.0 / (Fd.x[3] - Fd.x[2])) : T(0);
    }
  }
  __syncthreads();
  if (MODE != 2) {
    // the faces' stencil-cell and face boosts, phi^6 and rotations in T, one
    // item per thread (each item's global loads and float64 conversions
    // would otherwise queue behind one thread per face)
    for (int q = tid; q < nface * 41; q += NT) {
      const int f = q < 5 * nface ? q / 5 : (q - 5 * nface) / 36;
      const FaceDesc& Fd = S.F[f];
      if (Fd.type < 0) continue;
      if (q < 5 * nface) {
        const int k = q % 5;
        Loc<T>* L = S.L + 5 * f;
        if (k == 4) {
          make_loc(L[4], Fd.v, Fd.al, Fd.cf);
        } else {
          const int zz = Fd.z[k];
          S.FT[f].c6k[k] = zz >= 0 ? (T)pow6(st.cf[zz]) : T(0);
          if (zz >= 0) make_loc(L[k], st.v + 3 * zz, st.al[zz], st.cf[zz]);
        }
      } else {
        const int e = (q - 5 * nface) % 36, k = e / 9, m = e % 9;
        S.Gs[36 * f + e] = Fd.G[k] ? (T)Fd.G[k][m] : T(m % 4 == 0 ? 1 : 0);
      }
    }
    __syncthreads();
  }
  const T* P3 = S.p3 + NE + 1;       // P3[k] = R^(3k)

  // stencil rows of (face fi, species si) into SRC: bulk copies by thread 0
  auto issue = [&](int fi, int si) {
    if (!use_tma || tid != 0) return;
    const FaceDesc& Fn = S.F[fi];
    unsigned bytes = 0;
    for (int k = 0; k < 4; ++k) if (Fn.z[k] >= 0) bytes += rowbytes;
    fence_proxy_async();
    mbar_expect_tx(S.bar, bytes);
    for (int k = 0; k < 4; ++k)
      if (Fn.z[k] >= 0) tma_load_1d(SRC + k * nbin, fin + ((size_t)si * tb.n_zone + Fn.z[k]) * nbin, rowbytes, S.bar);
  };
  // next existing face after fi (or nface)
  auto next_face = [&](int fi) {
    int f = fi + 1;
    while (f < nface && S.F[f].type < 0) ++f;
    return f;
  };
  int first = MODE == 2 ? nface : next_face(-1);
  if (first < nface) issue(first, 0);

  for (int fidx = first; MODE != 2 && fidx < nface; fidx = next_face(fidx)) {
    const FaceDesc& F = S.F[fidx];
    const FaceT<T>& ft = S.FT[fidx];
    // deposits: into this zone's side(s) (fused), or both sides (face pass)
    const bool depP = MODE == 1 ? F.z[1] >= 0 : (F.own & 1) != 0;
    const bool depQ = MODE == 1 ? F.z[2] >= 0 : (F.own & 2) != 0;
    unsigned mask = 0;
    for (int k = 0; k < 4; ++k) if (F.z[k] >= 0) mask |= 1u << k;
    if (depP) mask |= 1u << 4;
    if (depQ) mask |= 1u << 5;

    // --- weights of the six remaps: slots 0..3 -> face, face -> slot 1, face -> slot 2
    const Loc<T>* LF = S.L + 5 * fidx;
    const T* GF = S.Gs + 36 * fidx;
    const EBr<T> Rg = make_ebr<T>((T)tb.R);
    {
      const Loc<T> Ls = LF[4];
      for (int q = tid; q < 6 * NA; q += NT) {
        int r = q / NA, ang = q % NA;
        if (!((mask >> r) & 1u)) continue;
        int slot = r < 4 ? r : r - 3;
        const T* G = F.G[slot] ? GF + 9 * slot : nullptr;
        Wt<T> w;
        if (sizeof(T) == 4 && st.sur_tab) {
          // learned remap: the table row of (zone, face fidx, remap r)
          w = reinterpret_cast<const Wt<T>*>(st.sur_tab)[((size_t)zone * kSurKindsAll + 1 + 6 * fidx + r) * NA + ang];
        } else {
          // one call site for both directions (cell -> face, face -> cell)
          const bool back = r >= 4;
          chain_weights(tb, S.mu, S.n0, S.n1, S.n2, back ? Ls : LF[slot], back ? LF[slot] : Ls, G, back ? 1 : 0,
                        F.axis, ang, Rg, w);
        }
        S.W[r * NA + ang] = w;
      }
      // face opacities and flux-switch weights per species and group
      // [R-10, R-12b], all species at once: their loads overlap the weights'
      // arithmetic instead of stalling each species' start
      if (F.type == F_INTERNAL) {
        for (int q = tid; q < NS * NE; q += NT) {
          const int sq = q / NE, i = q % NE;
          size_t oP = ((size_t)sq * tb.n_zone + F.z[1]) * NE + i;
          size_t oQ = ((size_t)sq * tb.n_zone + F.z[2]) * NE + i;
          double kaP = st.ka[oP], kaQ = st.ka[oQ], ksP = st.ks[oP], ksQ = st.ks[oQ];
          S.kaS[q] = (T)(0.5 * (kaP + kaQ));
          S.ksS[q] = (T)(0.5 * (ksP + ksQ));
          S.feS[q] = (T)(0.5 * (st.fe[oP] + st.fe[oQ]));
          S.wP[q] = exp_t((T)(-(kaP + ksP)) * ft.dx);
          S.wQ[q] = exp_t((T)(-(kaQ + ksQ)) * ft.dx);
        }
      }
      // face bins: Eulerian energy factor and normal coordinate velocity
      for (int ang = tid; ang < NA; ang += NT) {
        T n[3] = {S.n0[ang], S.n1[ang], S.n2[ang]};
        T e, p[3];
        boost_fwd(Ls, n, e, p);
        S.u0s[ang] = e;
        T vn = Ls.al / (Ls.cf * Ls.cf) * p[F.axis] / e;
        S.vns[ang] = vn;
        S.cs[ang] = T(1) / (ft.c6 * e * S.dOm[ang]);
        S.taus[ang] = T(0.5) * ft.dt * ft.al / e;
        S.vdx[ang] = T(0.5) * ft.dt * vn * ft.rdx;
      }
    }
    __syncthreads();
    // energy-pass parameters of this thread's column for the six remaps,
    // and the density factor of its angle for the four stencil cells
    int em[6];
    T ew[6], cang[4];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      if (gact && ((mask >> r) & 1u)) { em[r] = S.W[r * NA + gb].m; ew[r] = S.W[r * NA + gb].we; }
      else { em[r] = 0; ew[r] = T(0); }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      cang[k] = T(0);
      if (gact && F.z[k] >= 0) {
        const Loc<T>& Lk = LF[k];
        const T u0 = Lk.g * (T(1) + (Lk.v[0] * S.n0[gb] + Lk.v[1] * S.n1[gb] + Lk.v[2] * S.n2[gb]));
        cang[k] = ft.c6k[k] * u0 * S.dOm[gb];
      }
    }
    build_alists(S.W, 6, mask, NA, NMU, NPH, S.off, S.msk, S.ent);   // synchronises

    for (int s = 0; s < NS; ++s) {
      // this species' face opacities and flux-switch weights
      const T* kaS = S.kaS + (size_t)s * NE;
      const T* ksS = S.ksS + (size_t)s * NE;
      const T* feS = S.feS + (size_t)s * NE;
      const T* wPs = S.wP + (size_t)s * NE;
      const T* wQs = S.wQ + (size_t)s * NE;
      // stencil rows of this species (f as stored)
      if (use_tma) {
        bool ok = mbar_wait(S.bar, tphase, st.flag);
        tphase ^= 1u;
        if (__syncthreads_or(!ok)) {
          // give the copy in flight a second bounded chance, then stop
          if (tid == 0) mbar_wait(S.bar, tphase ^ 1u, st.flag);
          __syncthreads();
          return;
        }
      } else {
        if (gact) {
          for (int k = 0; k < 4; ++k) {
            const int zz = F.z[k];
            if (zz < 0) continue;
            const T* fz = fin + ((size_t)s * tb.n_zone + zz) * nbin;
            for (int i = gc; i < NE; i += nch) SRC[k * nbin + i * NA + gb] = fz[i * NA + gb];
          }
        }
        __syncthreads();
      }
      // energy pass of the stencil remaps (content density folded in)
      // (float32: one copy of the pass for the four cells, not four, so the
      // kernel body stays smaller and its instruction fetch stalls less;
      // float64, whose float64 pipe is the bound, keeps the four copies)
      if (gact) {
        if constexpr (sizeof(T) == 4) {
          // the four cells in one walk of the rows
          unsigned act = 0;
          for (int slot = 0; slot < 4; ++slot)
            if (F.z[slot] >= 0 && (F.type == F_INTERNAL || slot == 1 || slot == 2)) act |= 1u << slot;
          const T* srcs[4] = {SRC, SRC + nbin, SRC + 2 * nbin, SRC + 3 * nbin};
          T* outs[4] = {EB, EB + ebs, EB + 2 * ebs, EB + 3 * ebs};
          energy_cells<4, T, T>(gc, nch, NE, NA, gb, act, em, ew, cang, srcs, outs, rpt, P3);
        } else {
#pragma unroll
          for (int slot = 0; slot < 4; ++slot)
            if (F.z[slot] >= 0 && (F.type == F_INTERNAL || slot == 1 || slot == 2))
              energy_column<T, T, true>(gc, nch, NE, NA, gb, em[slot], ew[slot], SRC + slot * nbin, EB + slot * ebs,
                                        rpt, cang[slot], P3);
        }
      }
      __syncthreads();
      // angular pass: g_k = T_{k->s}[n_k] as face distribution (into SRC)
      if (gact) {
        const T csb = S.cs[gb];
        // the outer stencil cells feed only the upwind slope: P-1 where the
        // bin moves P -> Q, Q+1 where it moves Q -> P, and only at interior
        // faces; the other values are never read
        // (one pass serves both outer cells: each lane takes the one its bin
        // needs, so the warp does not run the two as separate passes)
        const bool upb = S.vns[gb] >= T(0);
#pragma unroll 1
        for (int k = 0; k < 3; ++k) {
          const int slot = k == 0 ? (upb ? 0 : 3) : k;
          if (F.z[slot] < 0) continue;
          if (k == 0 && F.type != F_INTERNAL) continue;
          const short* off = S.off + slot * (NA + 1);
          // (both outer cells' values go to the first row: each bin reads one)
          StoreG<T> st_g{SRC + k * nbin, csb, NA, gb};
          angular_rows<T, T, RB>(gc, nch, NE, NA, rpt, off[gb], off[gb + 1], S.ent + slot * alist_block(NA), EB + slot * ebs, st_g);
        }
      }
      __syncthreads();
      if (tb.pole) {
        // pole nodes of the remapped stencil values: rows of the cells P and
        // Q, and of the outer cell the node's flow direction reads (the same
        // for all of a pole node's cells: they share one direction)
        for (int q = tid; q < 6 * NE; q += NT) {
          const int k = q / (2 * NE), side = (q / NE) & 1, t = q % NE;
          const int j = side ? NMU - 1 : 0;
          const int slot = k == 0 ? (S.vns[j * NPH] >= T(0) ? 0 : 3) : k;
          if (F.z[slot] < 0 || (k == 0 && F.type != F_INTERNAL)) continue;
          T* c = SRC + k * nbin + t * NA + j * NPH;
          T sum = T(0);
          for (int kk = 0; kk < NPH; ++kk) sum += c[kk];
          sum = sum / T(NPH);
          for (int kk = 0; kk < NPH; ++kk) c[kk] = sum;
        }
        __syncthreads();
      }
      const T* G0 = SRC;          // the outer stencil cell each bin's upwind side reads
      const T* G1 = SRC + nbin;
      const T* G2 = SRC + 2 * nbin;
      T* RD = EB;                 // r / D
      T* FL = EB + ebs;           // flux content
      T* ID = EB + 2 * ebs;       // 1 / D
      // Lax-Wendroff half step with implicit collision [R-10]: per bin
      // r = (g1+g2)/2 - (dt/2) v (g2-g1)/dx + tau ka feq, D = 1 + (ka+ks) tau
      if (F.type == F_INTERNAL) {
        if (gact) {
          const T tau = S.taus[gb], vdx = S.vdx[gb];
          for (int i = gc; i < NE; i += nch) {
            const int q = i * NA + gb;
            const T g1 = G1[q], g2 = G2[q];
            const T r = T(0.5) * (g1 + g2) - vdx * (g2 - g1) + tau * kaS[i] * feS[i];
            const T iD = T(1) / (T(1) + (kaS[i] + ksS[i]) * tau);
            RD[q] = r * iD;
            ID[q] = iD;
          }
        }
        __syncthreads();
        // J per group (Sherman-Morrison closed form).  float32: one half-warp
        // per row (12 rows fill 256 threads in one round, every lane busy on
        // 80 angles); float64: one warp per row.  Either way the order of the
        // row sums does not depend on the launch shape.
        if constexpr (sizeof(T) == 4) {
          const int hw = tid >> 4, hl = tid & 15;
          for (int i0 = 0; i0 < NE; i0 += NT / 16) {
            const int i = i0 + hw;
            T sr = T(0), s1 = T(0);
            if (i < NE) {
              const T ka = kaS[i];
              for (int ang = hl; ang < NA; ang += 16) {
                const int q = i * NA + ang;
                const T dom = S.dOm[ang];
                sr += dom * RD[q];
                s1 += dom * ID[q] * (T(1) + ka * S.taus[ang]);
              }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
              sr += __shfl_down_sync(0xffffffffu, sr, o, 16);
              s1 += __shfl_down_sync(0xffffffffu, s1, o, 16);
            }
            if (hl == 0 && i < NE) S.rowJ[i] = sr / s1;
          }
        } else {
          for (int i = warp; i < NE; i += (NT / 32)) {
            T sr = T(0), s1 = T(0);
            const T ka = kaS[i];
            for (int ang = lane; ang < NA; ang += 32) {
              const int q = i * NA + ang;
              const T dom = S.dOm[ang];
              sr += dom * RD[q];
              s1 += dom * ID[q] * (T(1) + ka * S.taus[ang]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              sr += __shfl_down_sync(0xffffffffu, sr, o);
              s1 += __shfl_down_sync(0xffffffffu, s1, o);
            }
            if (lane == 0) S.rowJ[i] = sr / s1;
          }
        }
        __syncthreads();
      }
      // interface state (blend of LW and MC upwind) and flux content per face bin
      ff sumF = ff{0.0f, 0.0f};
      double tn = 0.0, te = 0.0;
      const bool outflow = F.type == F_OUTFLOW_P || F.type == F_OUTFLOW_Q;
      if (gact) {
        const T vn = S.vns[gb];
        const T fang = ft.dt * ft.area * ft.c6 * S.u0s[gb] * vn * S.dOm[gb];
        const int jj = gb / NPH, kk = gb % NPH;
        const int gm = (NMU - 1 - jj) * NPH + kk;   // mirror angle (reflecting wall)
        const bool up = vn >= T(0);
        const T taug = S.taus[gb];
        // the upwind side's constants (P where the bin moves P -> Q, else
        // Q), chosen once: the row loop then has no branch on the side, which
        // differs between the lanes of a warp
        const T rdlo = up ? ft.rdl0 : ft.rdl2;     // 1 / distance to the outer cell
        const T sup = up ? ft.sP : ft.sQ;          // distance cell -> face
        const T* wup = up ? wPs : wQs;             // flux-switch weights
        const bool has_outer = up ? F.z[0] >= 0 : F.z[3] >= 0;
        for (int i = gc; i < NE; i += nch) {
          const int q = i * NA + gb;
          T fs;
          if (F.type == F_INTERNAL) {
            const T g1 = G1[q], g2 = G2[q], go = G0[q];
            const T flw = RD[q] + ksS[i] * S.rowJ[i] * taug * ID[q];
            // MC-limited slope of the upwind cell (symmetric in its two
            // differences; no slope next to the grid's edge)
            const T od = (up ? g1 - go : go - g2) * rdlo;
            const T sl = has_outer ? mc_limiter(od, (g2 - g1) * ft.rdl1) : T(0);
            const T fu = (up ? g1 : g2) + sl * sup;
            const T w = wup[i];
            fs = (T(1) - w) * flw + w * fu;
          } else if (F.type == F_OUTFLOW_P) {
            // incoming bins: vacuum, or the distribution imposed on the open
            // face at theta_max [R-15b]
            fs = up ? G1[q] : (F.bc ? (T)st.fbc[((size_t)s * tb.n_r + a) * NE + i] : T(0));
          } else if (F.type == F_OUTFLOW_Q) {
            fs = vn < T(0) ? G2[q] : T(0);
          } else {  // reflecting wall at rest
            fs = vn < T(0) ? G2[q] : G2[i * NA + gm];
          }
          const T Fc = fang * fs;            // flux content per unit dGamma
          FL[q] = Fc;
          if (sizeof(T) == 4) sumF = ff_add(sumF, two_prod((float)Fc, (float)S.dGam[i]));
        }
        if (outflow) {
          const double sg = F.type == F_OUTFLOW_P ? 1.0 : -1.0;
          for (int i = gc; i < NE; i += nch) {
            double c = sg * (double)FL[i * NA + gb] * tb.dGam[i];
            tn += c;
            te += c * tb.eps[i] * (double)S.u0s[gb];
          }
        }
      }
      // the block's exact flux total, needed by one thread only: warp sums
      // now, their sum after the barrier the deposits need anyway.  In the
      // face pass that thread is the block's last (with the records below):
      // thread 0 also issues the next stencil copies, and the two serial
      // parts on one warp delayed the block's next barrier (face pass -2 to
      // -3.5 %)
      if (sizeof(T) == 4) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sumF = ff_add(sumF, ff_shfl_down(sumF, o));
        if (lane == 0) S.redf[warp] = sumF;
      }
      __syncthreads();
      constexpr int kTot = MODE == 1 ? NT - 1 : 0;   // the thread forming the total
      if (sizeof(T) == 4 && tid == kTot) {
        ff t = S.redf[0];
        for (int w = 1; w < NT / 32; ++w) t = ff_add(t, S.redf[w]);
        sumF = t;
      }
      // the stencil buffers are free: prefetch the next rows while depositing
      {
        int fn = fidx, sn = s + 1;
        if (sn == NS) { fn = next_face(fidx); sn = 0; }
        if (fn < nface) issue(fn, sn);
      }
      if (MODE == 0 && tid == 0 && sizeof(T) == 4) {
        // exact total of this zone's deposits: (+sum F if own Q) - (sum F if own P)
        if (F.own & 2) S.dtot[s] = ff_add(S.dtot[s], sumF);
        if (F.own & 1) S.dtot[s] = ff_add(S.dtot[s], ff_neg(sumF));
      }
      // outflow tallies (number and energy at infinity)
      double tn_sum = 0.0, te_sum = 0.0;
      if (outflow) {
        tn_sum = block_sum2(tn, te, S.red, te_sum);
        if (MODE == 0 && tid == 0) { S.tally[2 * s] += tn_sum; S.tally[2 * s + 1] += te_sum * F.al; }
      }
      if (MODE == 1 && tid == kTot) {
        // the receiving zones' records of this face: exact totals and tallies
        const ff zero = ff{0.0f, 0.0f};
        if (depP) {
          DepRec& r = rec[((size_t)F.z[1] * 6 + 2 * F.axis + 1) * NS + s];
          const ff sv = sizeof(T) == 4 ? ff_neg(sumF) : zero;
          if (F.addP) {
            r.sum = ff_add(r.sum, sv); r.tn += tn_sum; r.te += te_sum * F.al;
          } else {
            r.sum = sv; r.tn = tn_sum; r.te = te_sum * F.al;
          }
        }
        if (depQ) {
          DepRec& r = rec[((size_t)F.z[2] * 6 + 2 * F.axis) * NS + s];
          const ff sv = sizeof(T) == 4 ? sumF : zero;
          const double tnv = depP ? 0.0 : tn_sum, tev = depP ? 0.0 : te_sum * F.al;
          if (F.addQ) {
            r.sum = ff_add(r.sum, sv); r.tn += tnv; r.te += tev;
          } else {
            r.sum = sv; r.tn = tnv; r.te = tev;
          }
        }
      }
      // deposits into this zone: dN -= T_{s->P}[F] (own P), dN += T_{s->Q}[F] (own Q)
      T* EP = EB + 2 * ebs;
      T* EQ = EB + 3 * ebs;
      // both sides in one walk of the rows (float32), or one code path for
      // both sides (P first): a smaller kernel body
      if (gact) {
        if constexpr (sizeof(T) == 4) {
          const unsigned act = (depP ? 1u : 0u) | (depQ ? 2u : 0u);
          const T ones[2] = {T(1), T(1)};
          const T* srcs[2] = {FL, FL};
          T* outs[2] = {EP, EQ};
          energy_cells<2, T, T>(gc, nch, NE, NA, gb, act, em + 4, ew + 4, ones, srcs, outs, rpt, P3);
        } else {
#pragma unroll 1
          for (int side = 0; side < 2; ++side)
            if (side == 0 ? depP : depQ)
              energy_column<T, T, true>(gc, nch, NE, NA, gb, side == 0 ? em[4] : em[5], side == 0 ? ew[4] : ew[5], FL,
                                        side == 0 ? EP : EQ, rpt, T(1), P3);
        }
      }
      __syncthreads();
      if (gact) {
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          if (!(side == 0 ? depP : depQ)) continue;
          const short* off = S.off + (4 + side) * (NA + 1);
          const AList<T> ent = S.ent + (4 + side) * alist_block(NA);
          const T* Es = side == 0 ? EP : EQ;
          const T sgn = side == 0 ? T(-1) : T(1);
          if (MODE == 0) {
            angular_rows<T, T, RB>(gc, nch, NE, NA, rpt, off[gb], off[gb + 1], ent, Es,
                               AddDN<T>{S.dN + (size_t)s * nbin, NA, gb, sgn});
          } else {
            T* d = dep + (((size_t)F.z[1 + side] * 6 + 2 * F.axis + (side == 0 ? 1 : 0)) * NS + s) * nbin;
            angular_rows<T, T, RB>(gc, nch, NE, NA, rpt, off[gb], off[gb + 1], ent, Es, StoreDep<T>{d, NA, gb, sgn, side == 0 ? F.addP != 0 : F.addQ != 0});
          }
        }
      }
      __syncthreads();
    }
  }

  if constexpr (MODE == 1) return;   // the face pass ends here
  if (MODE == 0 && tb.pole) {
    // pole nodes of the summed deposits (the even spread is linear, so one
    // mean of the sum equals the sum of the faces' means); before the mixed
    // path's exact-total correction, which then also covers its rounding
    pole_mean(S.dN, NS * NE, NA, NMU, NPH);
    __syncthreads();
  }
  DN* dNall = S.dN;
  if constexpr (MODE == 2) {
    // gather this zone's deposits in the fused kernel's order: faces in
    // order; per face the rows P side then Q side, the exact totals Q side
    // then P side
    int rows[8], nrow = 0;   // this zone's deposit slots in that order
    for (int fidx = 0; fidx < nface; ++fidx) {
      if (!face_exists(tb, a, b, fidx)) continue;
      const int axis = fidx < 2 ? 0 : (fidx < 4 ? 1 : 2);
      const bool isP = fidx == 1 || fidx == 3 || fidx == 4 || (fidx == 2 && tb.periodic_th);
      const bool isQ = fidx == 0 || fidx == 4 || (fidx == 2);
      if (isP) rows[nrow++] = 2 * axis + 1;
      if (isQ) rows[nrow++] = 2 * axis;
    }
    // the sums go to the zone's first slot: each element is written by the
    // thread that has just read all of its rows, and no other zone reads
    // this zone's slots (the next face pass rewrites them before they are
    // read again), so shared memory holds no species-sized rows and more
    // CTAs fit on an SM
    dNall = dep + ((size_t)zone * 6 + rows[0]) * NS * nbin;
    // exact totals and outflow tallies of the zone's records
    if (warp == 0) zone_records(tb, rec, zone, a, b, nface, NS, sizeof(T) == 4, S.dtot, S.tally);
    // all of an element's rows are loaded before they are summed in order
    auto gather = [&](const T* base, int q) {
      T v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < nrow) v[k] = base[(size_t)rows[k] * NS * nbin + q];
      DN acc = DN(0);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < nrow) acc += (DN)v[k];
      return acc;
    };
    if (tb.pole) {
      // pole nodes: gather all species, spread the pole nodes' sums evenly
      // (as the fused kernel does), then find the correction below
      for (int s = 0; s < NS; ++s) {
        const T* base = dep + ((size_t)zone * 6 * NS + s) * nbin;
        DN* dNs = dNall + (size_t)s * nbin;
        for (int q = tid; q < nbin; q += NT) dNs[q] = gather(base, q);
      }
      __syncthreads();
      pole_mean(dNall, NS * NE, NA, NMU, NPH);
      __syncthreads();
    }
    for (int s = 0; s < NS; ++s) {
      // the mixed path's exact-total correction is found in the gathering
      // pass (or, with pole nodes, in a pass over the spread sums)
      const T* base = dep + ((size_t)zone * 6 * NS + s) * nbin;
      DN* dNs = dNall + (size_t)s * nbin;
      ff part = ff{0.0f, 0.0f};
      float bk = -1.0f;
      int bi = 0x7fffffff;
      auto tally = [&](int q, DN acc) {
        if (sizeof(T) == 4) {
          const float c = (float)acc * (float)S.dGam[q / NA];
          part = ff_add(part, two_prod((float)acc, (float)S.dGam[q / NA]));
          const float k = fabsf(c);
          if (k > bk) { bk = k; bi = q; }
        }
      };
      // with the grid fixed at compile time, two elements a thread per pass,
      // all of their rows loaded before either is summed (twice the loads
      // in flight; the generic kernel has no registers for them); each
      // thread still tallies its elements in ascending order
      for (int q0 = tid; q0 < nbin; q0 += kPair ? 2 * NT : NT) {
        const int q1 = q0 + NT;
        const bool has1 = kPair && q1 < nbin;
        DN acc0, acc1 = DN(0);
        if (tb.pole) {
          acc0 = dNs[q0];
          if (has1) acc1 = dNs[q1];
        } else {
          T v0[8], v1[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (k < nrow) {
              v0[k] = base[(size_t)rows[k] * NS * nbin + q0];
              v1[k] = has1 ? base[(size_t)rows[k] * NS * nbin + q1] : T(0);
            }
          }
          acc0 = DN(0);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k < nrow) { acc0 += (DN)v0[k]; acc1 += (DN)v1[k]; }
          dNs[q0] = acc0;
          if (has1) dNs[q1] = acc1;
        }
        tally(q0, acc0);
        if (has1) tally(q1, acc1);
      }
      if (sizeof(T) == 4) {
        // warp reductions now; the block's, for every species, after one
        // barrier below (same order of operations as a block reduction)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          part = ff_add(part, ff_shfl_down(part, o));
          const float k2 = __shfl_down_sync(0xffffffffu, bk, o);
          const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
          if (k2 > bk || (k2 == bk && i2 < bi)) { bk = k2; bi = i2; }
        }
        if (lane == 0) {
          S.redfS[s * kMaxWarps + warp] = part;
          S.rkeyS[s * kMaxWarps + warp] = bk;
          S.ridxS[s * kMaxWarps + warp] = bi;
        }
      }
    }
    __syncthreads();
    if (sizeof(T) == 4) {
      for (int s = tid; s < NS; s += NT) {
        ff tot = S.redfS[s * kMaxWarps];
        float kb = S.rkeyS[s * kMaxWarps];
        int at = S.ridxS[s * kMaxWarps];
        for (int w = 1; w < NT / 32; ++w) {
          tot = ff_add(tot, S.redfS[s * kMaxWarps + w]);
          const float k2 = S.rkeyS[s * kMaxWarps + w];
          const int i2 = S.ridxS[s * kMaxWarps + w];
          if (k2 > kb || (k2 == kb && i2 < at)) { kb = k2; at = i2; }
        }
        ff c = ff_add(S.dtot[s], ff_neg(tot));
        S.corr[s] = ff_to_d(c) / tb.dGam[at / NA];   // back to content per unit dGamma
        S.corr_f[s] = ff_from_d(S.corr[s]);
        S.corr_at[s] = at;
      }
      __syncthreads();
    }
  }

  // --- mixed path: restore the exact deposit total of every species before
  //     the collision (float accumulation rounds; number must not drift)
  if (sizeof(T) == 4 && MODE != 2) {   // (the zone pass found it while gathering)
    for (int s = 0; s < NS; ++s) {
      const DN* dNs = S.dN + (size_t)s * nbin;
      ff part = ff{0.0f, 0.0f};
      float bk = -1.0f;
      int bi = 0x7fffffff;
      for (int q = tid; q < nbin; q += NT) {
        const float c = (float)dNs[q] * (float)S.dGam[q / NA];
        part = ff_add(part, two_prod((float)dNs[q], (float)S.dGam[q / NA]));
        float k = fabsf(c);
        if (k > bk) { bk = k; bi = q; }
      }
      ff tot = block_sum_ff(part, S.redf);
      int at = block_argmax(bk, bi, S.rkey, S.ridx);
      if (tid == 0) {
        ff c = ff_add(S.dtot[s], ff_neg(tot));
        S.corr[s] = ff_to_d(c) / tb.dGam[at / NA];   // back to content per unit dGamma
        S.corr_f[s] = ff_from_d(S.corr[s]);
        S.corr_at[s] = at;
      }
    }
  } else if (sizeof(T) == 8) {
    for (int s = tid; s < NS; s += NT) { S.corr[s] = 0.0; S.corr_at[s] = -1; }
  }

  // --- implicit collision per (species, group) (Sec. 3.5) and moments (Eq. hydrosource)
  //     f* = f + dN / (phi^6 dV u0 dGamma dOmega); D_b = 1 + (ka+ks) tau_b,
  //     J = sum dOm r/D / sum dOm (1 + ka tau)/D, f = (r + ks tau J)/D
  // the zone's float64 scalars, formed once by one thread: float64 divisions
  // and square roots by every thread of the CTA would queue on GB300's
  // narrow float64 pipe
  if (tid == 0) {
    const double* v = st.v + 3 * zone;
    const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    S.zsc[0] = 1.0 / sqrt(1.0 - v2);       // gamma
    S.zsc[1] = st.al[zone];
    S.zsc[2] = pow6(st.cf[zone]);
    S.zsc[3] = 1.0 / (S.zsc[2] * tb.vol[zone]);
    S.zsc[4] = 1.0 / dt;
  }
  __syncthreads();
  const double gz = S.zsc[0], alz = S.zsc[1], c6z = S.zsc[2], rdt = S.zsc[4];
  {
    const double* v = st.v + 3 * zone;
    if constexpr (sizeof(T) == 8) {
      const double rcz = S.zsc[3];
      for (int ang = tid; ang < NA; ang += NT) {
        int j = ang / NPH, k = ang % NPH;
        double nv = v[0] * tb.mu[j] + (v[1] * tb.cph[k] + v[2] * tb.sph[k]) * tb.smu[j];
        double u0 = gz * (1.0 + nv);
        S.zu0[ang] = u0;
        S.ztau[ang] = alz * dt / u0;
        S.zcn[ang] = rcz / (u0 * tb.dOm[ang]);   // 1/(phi^6 dV u0 dOmega): dN is per unit dGamma
      }
    } else {
      // the mixed solve's per-angle constants in double-float: the two
      // reciprocals per angle by Newton steps on the FP32 pipes instead of
      // float64 divisions (GB300 runs float64 at 1/64 of the float32 rate)
      const ff alzdt = ff_from_d(alz * dt);
      const ff czone = ff_from_d(S.zsc[3]);
      // per-row opacity constants, converted once by one thread per row
      // (float64 work done by all 32 lanes of a row's warp costs 32x on the
      // narrow float64 pipe)
      for (int row = tid; row < NS * NE; row += NT) {
        const size_t oz = ((size_t)(row / NE) * tb.n_zone + zone) * NE + row % NE;
        const double ka = st.ka[oz], ks = st.ks[oz], fe = st.fe[oz];
        S.rowk[4 * row] = ff_from_d(ka);
        S.rowk[4 * row + 1] = ff_from_d(ks);
        S.rowk[4 * row + 2] = ff_from_d(ka + ks);
        S.rowk[4 * row + 3] = ff_from_d(ka * fe);
      }
      for (int ang = tid; ang < NA; ang += NT) {
        int j = ang / NPH, k = ang % NPH;
        double nv = v[0] * tb.mu[j] + (v[1] * tb.cph[k] + v[2] * tb.sph[k]) * tb.smu[j];
        double u0 = gz * (1.0 + nv);
        const ff ru0 = ff_recip(ff_from_d(u0));
        const ff dom = ff_from_d(tb.dOm[ang]);
        S.zt_f[ang] = ff_mul(alzdt, ru0);
        S.zc_f[ang] = ff_mul(ff_mul(czone, ru0), ff_recip(dom));   // dN is per unit dGamma
        S.zd_f[ang] = dom;
        S.zq_f[ang] = (float)(c6z * u0 * tb.dOm[ang] * rdt);
      }
    }
  }
  __syncthreads();
  for (int row = warp; row < NS * NE; row += (NT / 32)) {
    const int s = row / NE, i = row % NE;
    const T* fz = fin + ((size_t)s * tb.n_zone + zone) * nbin + (size_t)i * NA;
    const DN* dn = dNall + (size_t)s * nbin + (size_t)i * NA;
    const int cat = S.corr_at[s] - i * NA;       // corrected bin of this row, if any
    T* fo = fout + ((size_t)s * tb.n_zone + zone) * nbin + (size_t)i * NA;
    double mN = 0.0, mE = 0.0, mP0 = 0.0, mP1 = 0.0, mP2 = 0.0;
    int bad = 0;
    if constexpr (sizeof(T) == 8) {
      const size_t oz = ((size_t)s * tb.n_zone + zone) * NE + i;
      const double ka = st.ka[oz], ks = st.ks[oz], fe = st.fe[oz];
      const double cval = S.corr[s];
      const double cdg = c6z * tb.dGam[i] * rdt;
      const double kt = ka + ks, kafe = ka * fe;
      double* rr = S.wr_r + (size_t)warp * NA;
      double* ri = S.wr_i + (size_t)warp * NA;
      double sr = 0.0, s1 = 0.0;
      for (int ang = lane; ang < NA; ang += 32) {
        double tau = S.ztau[ang];
        double dnv = (double)dn[ang] + (ang == cat ? cval : 0.0);
        double fst = (double)fz[ang] + dnv * S.zcn[ang];
        double r = fst + tau * kafe;
        double iD = 1.0 / (1.0 + kt * tau);
        rr[ang] = fst;
        ri[ang] = iD;
        double dom = tb.dOm[ang];
        sr += dom * r * iD;
        s1 += dom * (1.0 + ka * tau) * iD;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      const double J = sr / s1;
      for (int ang = lane; ang < NA; ang += 32) {
        double tau = S.ztau[ang];
        double fst = rr[ang];
        double r = fst + tau * kafe;
        double fn = (r + ks * tau * J) * ri[ang];
        fo[ang] = (T)fn;
        bad |= !isfinite(fn);
        double dc = cdg * S.zu0[ang] * tb.dOm[ang] * (fn - fst);
        mN += dc;
        double de = dc * tb.eps[i];
        mE += de;
        mP0 += de * (double)S.n0[ang];
        mP1 += de * (double)S.n1[ang];
        mP2 += de * (double)S.n2[ang];
      }
    } else {
      // mixed path: double-float (about 48-bit) arithmetic on the FP32 pipes
      // keeps the solve conservative to well below 1e-10 where float32 would
      // not, at a fraction of GB300's float64 cost
      const ff ka_f = S.rowk[4 * row], ks_f = S.rowk[4 * row + 1];
      const ff kt_f = S.rowk[4 * row + 2], kafe_f = S.rowk[4 * row + 3];
      float* buf = reinterpret_cast<float*>(S.wr_r) + (size_t)warp * 4 * NA;   // fst.hi, fst.lo, iD.hi, iD.lo
      // per bin f* = f + zcn dN and 1/D; per row A = sum dOm f*/D,
      // B = sum dOm tau/D, C = sum dOm/D, so that sum dOm r/D = A + ka fe B
      // and sum dOm (1 + ka tau)/D = C + ka B
      ff sA = ff{0.0f, 0.0f}, sB = ff{0.0f, 0.0f}, sC = ff{0.0f, 0.0f};
      const ff cval_f = S.corr_f[s];
      auto bin1 = [&](int ang, float dnv, float fzv) {
        const ff tau = S.zt_f[ang];
        const ff zcn = S.zc_f[ang];
        const ff dom = S.zd_f[ang];
        ff p = ff_mul_f(zcn, dnv);
        if (ang == cat) p = ff_add(p, ff_mul(zcn, cval_f));
        const ff fst = ff_add(p, fzv);
        const ff iD = ff_recip(ff_add(ff_mul(kt_f, tau), 1.0f));
        buf[4 * ang] = fst.hi; buf[4 * ang + 1] = fst.lo;
        buf[4 * ang + 2] = iD.hi; buf[4 * ang + 3] = iD.lo;
        const ff w = ff_mul(dom, iD);
        sA = ff_add(sA, ff_mul(w, fst));
        sB = ff_add(sB, ff_mul(w, tau));
        sC = ff_add(sC, w);
      };
      // two angles a lane per pass, both loaded first (in ascending order)
      for (int a0 = lane; a0 < NA; a0 += 64) {
        const int a1 = a0 + 32;
        const bool has1 = a1 < NA;
        const float d0 = (float)dn[a0], f0 = (float)fz[a0];
        const float d1 = has1 ? (float)dn[a1] : 0.0f, f1 = has1 ? (float)fz[a1] : 0.0f;
        bin1(a0, d0, f0);
        if (has1) bin1(a1, d1, f1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sA = ff_add(sA, ff_shfl_xor(sA, o));
        sB = ff_add(sB, ff_shfl_xor(sB, o));
        sC = ff_add(sC, ff_shfl_xor(sC, o));
      }
      const ff sr = ff_add(sA, ff_mul(kafe_f, sB));
      const ff s1 = ff_add(sC, ff_mul(ka_f, sB));
      const ff J = ff_mul(sr, ff_recip(s1));
      // f = (f* + tau (ka fe + ks J)) / D
      const ff gJ = ff_add(kafe_f, ff_mul(ks_f, J));
      // number and momentum weights of the row; energy is eps_i times them
      float fN = 0.0f, fP0 = 0.0f, fP1 = 0.0f, fP2 = 0.0f;
      const float eps_i = (float)S.epsS[i];
      const float dg_i = (float)S.dGam[i];
      for (int ang = lane; ang < NA; ang += 32) {
        const ff tau = S.zt_f[ang];
        const ff fst = ff{buf[4 * ang], buf[4 * ang + 1]};
        const ff iD = ff{buf[4 * ang + 2], buf[4 * ang + 3]};
        const ff fn = ff_mul(ff_add(fst, ff_mul(tau, gJ)), iD);
        const float fw = fn.hi + fn.lo;
        fo[ang] = fw;
        bad |= !isfinite(fw);
        const ff del = ff_add(ff_neg(fst), fw);
        const float dc = S.zq_f[ang] * dg_i * (del.hi + del.lo);
        fN += dc;
        fP0 += dc * (float)S.n0[ang];
        fP1 += dc * (float)S.n1[ang];
        fP2 += dc * (float)S.n2[ang];
      }
      // the lane sums are float32 already: reduce them in float32 too
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        fN += __shfl_xor_sync(0xffffffffu, fN, o);
        fP0 += __shfl_xor_sync(0xffffffffu, fP0, o);
        fP1 += __shfl_xor_sync(0xffffffffu, fP1, o);
        fP2 += __shfl_xor_sync(0xffffffffu, fP2, o);
      }
      if (lane == 0) {   // float32 row partials; summed per species below
        float* zf = reinterpret_cast<float*>(S.zrow) + (size_t)row * 5;
        zf[0] = fN; zf[1] = fN * eps_i; zf[2] = fP0 * eps_i; zf[3] = fP1 * eps_i; zf[4] = fP2 * eps_i;
      }
    }
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mN += __shfl_xor_sync(0xffffffffu, mN, o);
        mE += __shfl_xor_sync(0xffffffffu, mE, o);
        mP0 += __shfl_xor_sync(0xffffffffu, mP0, o);
        mP1 += __shfl_xor_sync(0xffffffffu, mP1, o);
        mP2 += __shfl_xor_sync(0xffffffffu, mP2, o);
      }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if constexpr (sizeof(T) == 8) {
        double* zr = S.zrow + (size_t)row * 5;
        zr[0] = mN; zr[1] = mE; zr[2] = mP0; zr[3] = mP1; zr[4] = mP2;
      }
      if (bad) st.flag[0] = 1;
    }
  }
  __syncthreads();
  for (int s = tid; s < NS; s += NT) {
    double m[5] = {0, 0, 0, 0, 0};
    if constexpr (sizeof(T) == 8) {
      for (int i = 0; i < NE; ++i)
        for (int c = 0; c < 5; ++c) m[c] += S.zrow[((size_t)s * NE + i) * 5 + c];
    } else {
      // double-float sums of the float32 row partials, converted once
      const float* zf = reinterpret_cast<const float*>(S.zrow);
      ff acc[5] = {ff{0.0f, 0.0f}, ff{0.0f, 0.0f}, ff{0.0f, 0.0f}, ff{0.0f, 0.0f}, ff{0.0f, 0.0f}};
      for (int i = 0; i < NE; ++i)
        for (int c = 0; c < 5; ++c) acc[c] = ff_add(acc[c], zf[((size_t)s * NE + i) * 5 + c]);
      for (int c = 0; c < 5; ++c) m[c] = ff_to_d(acc[c]);
    }
    size_t o = (size_t)s * tb.n_zone + zone;
    if (lts) {
      // local time stepping: the zone's steps add up to the macro step's
      // moments (averaged over the macro step) and outflow
      const double sc = dt / (st.dt0 * (double)(1 << (st.lts_L - 1)));
      for (int c = 0; c < 5; ++c) m[c] *= sc;
      st.mom_N[o] += m[0];
      st.mom_E[o] += m[1];
      st.mom_P[3 * o] += m[2]; st.mom_P[3 * o + 1] += m[3]; st.mom_P[3 * o + 2] += m[4];
      st.out_N[o] += S.tally[2 * s];
      st.out_E[o] += S.tally[2 * s + 1];
    } else {
      st.mom_N[o] = m[0];
      st.mom_E[o] = m[1];
      st.mom_P[3 * o] = m[2]; st.mom_P[3 * o + 1] = m[3]; st.mom_P[3 * o + 2] = m[4];
      st.out_N[o] = S.tally[2 * s];
      st.out_E[o] = S.tally[2 * s + 1];
    }
    S.corr[s] = m[0];   // the species' number source (the correction is spent)
  }
  __syncthreads();
  if (tid == 0) {
    // Q_Ye = -(dN_nue - dN_nuebar) / h^3 (Eq. hydrosource)
    double q = 0.0;
    for (int s = 0; s < NS; ++s) {
      int kind = tb.species_kind[s];
      if (kind != 0 && kind != 1) continue;
      const double m = S.corr[s];
      q += kind == 0 ? -m : m;
    }
    if (lts) st.qye[zone] += q * st.phase_norm;
    else st.qye[zone] = q * st.phase_norm;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT >= 512 ? 1 : 768 / NT) : 1)
    k_flux_collide(Tables tb, State st, double dt) {
  flux_body<T, NT, 0>(tb, st, dt, nullptr, nullptr);
}
// the face pass keeps no dN or collision arrays: in float32 four 256-thread
// CTAs fit an SM (64 registers, no spills); 512-thread CTAs are for large
// rows, where shared memory allows one or two per SM anyway
// RB: rows per angular-list walk, chosen per problem by face_rb (the
// results do not depend on it: every row sums its list in the same order)
template <typename T, int NT, int RB = default_rb(NT), int NEC = 0, int NAC = 0, int NMUC = 0, int NPHC = 0>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? (NT >= 512 ? 2 : 1024 / NT) : 1)
    k_flux_faces(Tables tb, State st, double dt, T* dep, DepRec* rec) {
  flux_body<T, NT, 1, RB, NEC, NAC, NMUC, NPHC>(tb, st, dt, dep, rec);
}
template <typename T, int NEC = 0, int NAC = 0, int NMUC = 0, int NPHC = 0>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3) k_zone_collide(Tables tb, State st, double dt, T* dep, DepRec* rec) {
  flux_body<T, 256, 2, default_rb(256), NEC, NAC, NMUC, NPHC>(tb, st, dt, dep, rec);
}

// ---------------------------------------------------------------------------
// Time remap T_{n->n+1} of every zone (Sec. 3.2): old frames -> new frames
// ---------------------------------------------------------------------------
template <typename T>
struct RemapSmem {
  T* src[2];   // species rows (bulk copies; converted in place to content per dGamma), double-buffered
  T* E; T* dst; T* mu; T* n0; T* n1; T* n2; T* dOm; T* dGam; T* p3;
  Wt<T>* W; AList<T> ent; short* off; unsigned* msk;
  ff* redf; float* rkey; int* ridx;
  unsigned long long* bar;   // [2] mbarriers of the two row buffers
  Loc<T>* L;                 // [2] the old and the new background of the zone
  T* c6;                     // [2] their phi^6
};

template <typename T>
__host__ __device__ size_t remap_smem_layout(int ne, int nang, int nmu, int nt, RemapSmem<T>* s, unsigned char* base) {
  size_t o = 0;
#define BT_TAKE(ptr, type, count)                              \
  do {                                                         \
    o = (o + 15) & ~size_t(15);                                \
    if (s) s->ptr = reinterpret_cast<type*>(base + o);         \
    o += sizeof(type) * (size_t)(count);                       \
  } while (0)
  BT_TAKE(bar, unsigned long long, 2);
  BT_TAKE(src[0], T, (size_t)ne * nang);
  BT_TAKE(src[1], T, (size_t)ne * nang);
  {
    // the energy pass's output (chunk layout), over the weights and list
    // bitmasks, which are dead once the lists are built (a species' remapped
    // rows go back into its own source buffer: no third row buffer)
    o = (o + 15) & ~size_t(15);
    const size_t e_bytes = sizeof(T) * chunk_elems(ne, nang, nt, 4);
    const size_t w_bytes = (sizeof(Wt<T>) * (size_t)nang + 15) & ~size_t(15);
    const size_t m_bytes = sizeof(unsigned) * (size_t)nang * ((nang + 31) / 32);
    if (s) {
      s->E = reinterpret_cast<T*>(base + o);
      s->W = reinterpret_cast<Wt<T>*>(base + o);
      s->msk = reinterpret_cast<unsigned*>(base + o + w_bytes);
      s->dst = nullptr;
    }
    o += e_bytes > w_bytes + m_bytes ? e_bytes : w_bytes + m_bytes;
  }
  BT_TAKE(mu, T, nmu);
  BT_TAKE(n0, T, nang);
  BT_TAKE(n1, T, nang);
  BT_TAKE(n2, T, nang);
  BT_TAKE(dOm, T, nang);
  BT_TAKE(dGam, T, ne);
  BT_TAKE(p3, T, 2 * ne + 3);
  BT_TAKE(ent.w, T, alist_block(nang));
  BT_TAKE(ent.b, short, alist_block(nang));
  BT_TAKE(off, short, nang + 1);
  BT_TAKE(redf, ff, 4 * kWarps);     // [species parity][input, output total][warp]
  BT_TAKE(rkey, float, 2 * kWarps);  // [species parity][warp]
  BT_TAKE(ridx, int, 2 * kWarps);
  BT_TAKE(L, Loc<T>, 2);
  BT_TAKE(c6, T, 2);
#undef BT_TAKE
  return (o + 15) & ~size_t(15);
}

// The mixed path's exact-total correction of one species of a zone, by one
// warp: the input and output content totals and the largest output bin from
// the nw warps' partials (a shuffle tree); lane 0 rewrites that bin's f with
// the correction, so the zone's content after the remap equals the content
// before it exactly (float gathers round).
template <typename T>
__device__ void remap_correct(const Tables& tb, int nw, const ff* pin, const float* pk, const int* pi, const T* dst,
                              T* fz, const Loc<T>& Y, T c6y, const T* n0, const T* n1, const T* n2, const T* dOm) {
  const int lane = threadIdx.x & 31;
  ff tot_in = lane < nw ? pin[lane] : ff{0.0f, 0.0f};
  ff tot = lane < nw ? pin[kWarps + lane] : ff{0.0f, 0.0f};
  float kb = lane < nw ? pk[lane] : -2.0f;
  int at = lane < nw ? pi[lane] : 0x7fffffff;
  int o0 = 1;   // the first shuffle distance that reaches a warp's partial
  while (2 * o0 < nw) o0 *= 2;
  for (int o = o0; o > 0; o >>= 1) {
    tot_in = ff_add(tot_in, ff_shfl_down(tot_in, o));
    tot = ff_add(tot, ff_shfl_down(tot, o));
    const float k2 = __shfl_down_sync(0xffffffffu, kb, o);
    const int i2 = __shfl_down_sync(0xffffffffu, at, o);
    if (k2 > kb || (k2 == kb && i2 < at)) { kb = k2; at = i2; }
  }
  if (lane != 0 || at < 0 || at >= tb.n_e * tb.n_ang) return;
  const int NA = tb.n_ang, b = at % NA;
  // the correction is a rounding-level term: float arithmetic (no float64
  // division on the block's critical path) keeps it to well below f's own
  // rounding
  const ff dc = ff_add(tot_in, ff_neg(tot));
  const float corr_y = (dc.hi + dc.lo) * tb.f_rdGam[at / NA];
  const T u0 = Y.g * (T(1) + (Y.v[0] * n0[b] + Y.v[1] * n1[b] + Y.v[2] * n2[b]));
  const T rc = T(1) / (c6y * u0 * dOm[b]);
  fz[at] = (dst[at] + (T)corr_y) * rc;
}

// Time remap T_{n->n+1} of every zone (Sec. 3.2): old frames -> new frames,
// one CTA per zone, the species one after another.  The species' rows come
// by bulk asynchronous copies (the first while the weights and lists are
// built, the next while the current species is remapped).  Two block
// barriers per species: the energy pass reads other threads' rows of its
// column, the angular pass other columns.  The mixed path's exact-total
// correction of a species is made by one thread after the next barrier
// (every thread writes its bins first, uncorrected).
// NEC, NAC, NMUC, NPHC: the grid's group and angle counts at compile time (0: taken from tb)
template <typename T, int NT, int NEC = 0, int NAC = 0, int NMUC = 0, int NPHC = 0>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : 4) k_time_remap(Tables tb, State st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RemapSmem<T> S;
  const int NE = NEC ? NEC : tb.n_e, NA = NAC ? NAC : tb.n_ang, NS = tb.n_s;
  const int NPH = NPHC ? NPHC : tb.n_ph, NMU = NMUC ? NMUC : tb.n_mu;
  remap_smem_layout<T>(NE, NA, NMU, NT, &S, smem_raw);
  const int rpt = chunk_rpt(NE, NA, NT, 4);
  constexpr int NW = NT / 32;
  const int zone = blockIdx.x;
  const int nbin = NE * NA;
  const int tid = threadIdx.x;
  const int nch = NT / NA > 0 ? NT / NA : 1;
  const int gb = tid % NA, gc = tid / NA;
  const bool gact = tid < nch * NA;
  T* f = reinterpret_cast<T*>(st.f);
  const unsigned rowbytes = (unsigned)(sizeof(T) * (size_t)nbin);
  const bool use_tma = (rowbytes % 16u) == 0u;
  auto row = [&](int s) { return f + ((size_t)s * tb.n_zone + zone) * nbin; };
  // the first species' row, copied while the tables, weights and lists are built
  if (tid == 0) {
    mbar_init(S.bar, 1);
    mbar_init(S.bar + 1, 1);
    if (use_tma) {
      mbar_expect_tx(S.bar, rowbytes);
      tma_load_1d(S.src[0], row(0), rowbytes, S.bar);
    }
  } else if (tid == 32) {
    // the zone's old and new frames, once (float64 loads and conversions
    // by every thread would queue on the narrow float64 pipe)
    make_loc(S.L[0], st.v_old + 3 * zone, st.al_old[zone], st.cf_old[zone]);
    make_loc(S.L[1], st.v + 3 * zone, st.al[zone], st.cf[zone]);
    S.c6[0] = (T)pow6(st.cf_old[zone]);
    S.c6[1] = (T)pow6(st.cf[zone]);
  }
  if constexpr (sizeof(T) == 4) {
    for (int q = tid; q < NMU; q += NT) S.mu[q] = tb.f_mu[q];
    for (int q = tid; q < NA; q += NT) {
      S.n0[q] = tb.f_n0[q]; S.n1[q] = tb.f_n1[q]; S.n2[q] = tb.f_n2[q]; S.dOm[q] = tb.f_dOm[q];
    }
    for (int q = tid; q < NE; q += NT) S.dGam[q] = tb.f_dGam[q];
    for (int q = tid; q < 2 * NE + 3; q += NT) S.p3[q] = tb.f_p3[q];
  } else {
    for (int q = tid; q < NMU; q += NT) S.mu[q] = (T)tb.mu[q];
    for (int q = tid; q < NA; q += NT) {
      int j = q / NPH, k = q % NPH;
      S.n0[q] = (T)tb.mu[j];
      S.n1[q] = (T)(tb.smu[j] * tb.cph[k]);
      S.n2[q] = (T)(tb.smu[j] * tb.sph[k]);
      S.dOm[q] = (T)tb.dOm[q];
    }
    for (int q = tid; q < NE; q += NT) S.dGam[q] = (T)tb.dGam[q];
    for (int q = tid; q < 2 * NE + 3; q += NT) S.p3[q] = (T)tb.p3[q];
  }
  __syncthreads();
  const T* P3 = S.p3 + NE + 1;
  const Loc<T> X = S.L[0], Y = S.L[1];
  const EBr<T> Rg = make_ebr<T>((T)tb.R);
  for (int ang = tid; ang < NA; ang += NT) {
    if (sizeof(T) == 4 && st.sur_tab)
      S.W[ang] = reinterpret_cast<const Wt<T>*>(st.sur_tab)[(size_t)zone * kSurKindsAll * NA + ang];
    else
      chain_weights(tb, S.mu, S.n0, S.n1, S.n2, X, Y, (const T*)nullptr, 0, AX_TIME, ang, Rg, S.W[ang]);
  }
  __syncthreads();
  const int em = gact ? S.W[gb].m : 0;
  const T ew = gact ? S.W[gb].we : T(0);
  build_alists(S.W, 1, 1u, NA, NMU, NPH, S.off, S.msk, S.ent);
  const T c6x = S.c6[0], c6y = S.c6[1];
  // this thread's column: density factor of the old frame, reciprocal of the new one's
  T cangX = T(0), rcY = T(1);
  if (gact) {
    const T u0x = X.g * (T(1) + (X.v[0] * S.n0[gb] + X.v[1] * S.n1[gb] + X.v[2] * S.n2[gb]));
    const T u0y = Y.g * (T(1) + (Y.v[0] * S.n0[gb] + Y.v[1] * S.n1[gb] + Y.v[2] * S.n2[gb]));
    cangX = c6x * u0x * S.dOm[gb];
    rcY = T(1) / (c6y * u0y * S.dOm[gb]);
  }
  const int lane = tid & 31, warp = tid >> 5;
  unsigned ph0 = 0u, ph1 = 0u;   // parity of the next phase of each buffer's mbarrier
  for (int s = 0; s < NS; ++s) {
    T* fz = row(s);
    const bool odd = (s & 1) != 0;
    T* src = odd ? S.src[1] : S.src[0];
    ff* pin = S.redf + (s & 1) * 2 * kWarps;      // [0, kWarps): input total, then output total
    float* pk = S.rkey + (s & 1) * kWarps;
    int* pi = S.ridx + (s & 1) * kWarps;
    S.dst = src;   // this species' remapped rows, once the energy pass has read src
    if (use_tma) {
      unsigned long long* bar_cur = S.bar + (odd ? 1 : 0);
      bool ok = mbar_wait(bar_cur, odd ? ph1 : ph0, st.flag);
      if (odd) ph1 ^= 1u; else ph0 ^= 1u;
      if (__syncthreads_or(!ok)) {
        // give the copy in flight a second bounded chance to land, then stop
        // (the next species' copy is issued only after this one's energy pass)
        if (tid == 0) mbar_wait(bar_cur, odd ? (ph1 ^ 1u) : (ph0 ^ 1u), st.flag);
        __syncthreads();
        return;
      }
    }
    // content per unit dGamma of the old frame, y = phi^6 u0 dOmega f, in
    // place; the mixed path's input total
    ff part = ff{0.0f, 0.0f};
    if (gact) {
      for (int i = gc; i < NE; i += nch) {
        const int q = i * NA + gb;
        const T d = cangX * (use_tma ? src[q] : fz[q]);
        src[q] = d;
        if (sizeof(T) == 4) part = ff_add(part, two_prod((float)d, (float)S.dGam[i]));
      }
    }
    if (sizeof(T) == 4) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part = ff_add(part, ff_shfl_down(part, o));
      if (lane == 0) pin[warp] = part;
    }
    __syncthreads();
    // the last species' exact-total correction (its bins were all written
    // before the barrier), by one thread while the others go on
    if (sizeof(T) == 4 && s > 0 && warp == 0) {
      const int sp = s - 1;   // its remapped rows are in its own source buffer
      remap_correct<T>(tb, NW, S.redf + (sp & 1) * 2 * kWarps, S.rkey + (sp & 1) * kWarps, S.ridx + (sp & 1) * kWarps,
                       (sp & 1) ? S.src[1] : S.src[0], row(sp), Y, c6y, S.n0, S.n1, S.n2, S.dOm);
    }
    if (gact) energy_column<T, T>(gc, nch, NE, NA, gb, em, ew, src, S.E, rpt, T(1), P3);
    __syncthreads();
    // the next species' row into the other buffer: its last readers (the
    // previous species' output loop and correction) are done
    if (use_tma && tid == 0 && s + 1 < NS) {
      unsigned long long* bar_nxt = S.bar + (odd ? 0 : 1);
      fence_proxy_async();
      mbar_expect_tx(bar_nxt, rowbytes);
      tma_load_1d(odd ? S.src[0] : S.src[1], row(s + 1), rowbytes, bar_nxt);
    }
    // the remapped rows (this thread's own bins), with the mixed path's
    // partials of the output total and of the largest bin
    if (gact) angular_rows<T, T, 4>(gc, nch, NE, NA, rpt, S.off[gb], S.off[gb + 1], S.ent, S.E, StoreT<T>{S.dst, NA, gb});
    if (tb.pole) {
      __syncthreads();
      pole_mean(S.dst, NE, NA, NMU, NPH);
      __syncthreads();
    }
    ff partc = ff{0.0f, 0.0f};
    float bk = -1.0f;
    int bi = 0x7fffffff;
    if (gact) {
      for (int i = gc; i < NE; i += nch) {
        const int q = i * NA + gb;
        const T d = S.dst[q];
        if (sizeof(T) == 4) {
          partc = ff_add(partc, two_prod((float)d, (float)S.dGam[i]));
          const float k = fabsf((float)d * (float)S.dGam[i]);
          if (k > bk) { bk = k; bi = q; }
        }
        fz[q] = d * rcY;   // f in the new frame (the correction follows)
      }
    }
    if (sizeof(T) == 4) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        partc = ff_add(partc, ff_shfl_down(partc, o));
        const float k2 = __shfl_down_sync(0xffffffffu, bk, o);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        if (k2 > bk || (k2 == bk && i2 < bi)) { bk = k2; bi = i2; }
      }
      if (lane == 0) { pin[kWarps + warp] = partc; pk[warp] = bk; pi[warp] = bi; }
    }
  }
  if (sizeof(T) == 4) {
    __syncthreads();
    if (warp == 0) {
      const int sp = NS - 1;
      remap_correct<T>(tb, NW, S.redf + (sp & 1) * 2 * kWarps, S.rkey + (sp & 1) * kWarps, S.ridx + (sp & 1) * kWarps,
                       (sp & 1) ? S.src[1] : S.src[0], row(sp), Y, c6y, S.n0, S.n1, S.n2, S.dOm);
    }
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
  const double c6 = pow6(st.cf[zone]), al = st.al[zone], vol = tb.vol[zone];
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
__global__ void __launch_bounds__(kThreads) k_max_rate(Tables tb, State st, unsigned long long* out, double* zr) {
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
    if (zr) zr[zone] = mm;   // per-zone rate (levels of the local time stepping)
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

// ---------------------------------------------------------------------------
// Learned remap: the rows it predicts, their input features and the exact
// targets.  A row is (zone, kind, source angle).  kind 0 is the zone's time
// remap (previous -> current background, Sec. 3.2 with G = I); kind
// 1 + 6 fidx + r is remap r of the zone's face fidx (r < 4: stencil cell r ->
// face, r = 4, 5: face -> cell 1, 2; Sec. 3.3).
// ---------------------------------------------------------------------------

struct RemapRow {
  const double* vX;
  const double* vY;
  double alX, alY, cfX, cfY;
  const double* G;   // rotation passed to the chain (nullptr: none)
  int gT;            // chain applies G transposed
  int axis;
};

// false if the row's remap does not exist (no face, zero area, absent cell)
__device__ bool sur_row(const Tables& tb, const State& st, int zone, int kind, FaceDesc& F, RemapRow& R) {
  if (kind == 0) {
    R.vX = st.v_old + 3 * zone; R.alX = st.al_old[zone]; R.cfX = st.cf_old[zone];
    R.vY = st.v + 3 * zone; R.alY = st.al[zone]; R.cfY = st.cf[zone];
    R.G = nullptr; R.gT = 0; R.axis = AX_TIME;
    return true;
  }
  const int fidx = (kind - 1) / 6, r = (kind - 1) % 6;
  if (!make_face(tb, st, zone % tb.n_r, zone / tb.n_r, fidx, F)) return false;
  const int slot = r < 4 ? r : r - 3;
  const int z = F.z[slot];
  if (z < 0) return false;
  R.G = F.G[slot];
  R.axis = F.axis;
  if (r < 4) {
    R.vX = st.v + 3 * z; R.alX = st.al[z]; R.cfX = st.cf[z];
    R.vY = F.v; R.alY = F.al; R.cfY = F.cf;
    R.gT = 0;
  } else {
    R.vX = F.v; R.alX = F.al; R.cfX = F.cf;
    R.vY = st.v + 3 * z; R.alY = st.al[z]; R.cfY = st.cf[z];
    R.gT = 1;
  }
  return true;
}

// The 16 inputs of the network for row (R, source angle ang):
//  0-2   source direction n in the source triad
//  3-5   source fluid velocity (source triad)
//  6-8   destination fluid velocity expressed in the source triad, Gc^T v_Y
//  9-11  rotation vector of Gc (source -> destination triad), the
//        antisymmetric part (Gc - Gc^T)/2 as a vector
//  12-14 ln(alpha_X / alpha_Y) along the kick axis (zero for the time remap)
//  15    ln((phi_X / phi_Y)^2)
__device__ void sur_features(const Tables& tb, const RemapRow& R, int ang, double* f) {
  const int j = ang / tb.n_ph, k = ang % tb.n_ph;
  f[0] = tb.mu[j];
  f[1] = tb.smu[j] * tb.cph[k];
  f[2] = tb.smu[j] * tb.sph[k];
  double Gc[9];
  for (int m = 0; m < 3; ++m)
    for (int c = 0; c < 3; ++c)
      Gc[3 * m + c] = R.G ? (R.gT ? R.G[3 * c + m] : R.G[3 * m + c]) : (m == c ? 1.0 : 0.0);
  for (int c = 0; c < 3; ++c) {
    f[3 + c] = R.vX[c];
    f[6 + c] = Gc[c] * R.vY[0] + Gc[3 + c] * R.vY[1] + Gc[6 + c] * R.vY[2];
  }
  f[9] = 0.5 * (Gc[7] - Gc[5]);
  f[10] = 0.5 * (Gc[2] - Gc[6]);
  f[11] = 0.5 * (Gc[3] - Gc[1]);
  f[12] = f[13] = f[14] = 0.0;
  if (R.axis < 3) f[12 + R.axis] = log(R.alX / R.alY);
  f[15] = 2.0 * log(R.cfX / R.cfY);
}

// offset of a Phi index difference, wrapped to the nearest image
__device__ __forceinline__ int phi_offset(int d, int nph) {
  if (nph >= 3) {
    if (2 * d >= nph) d -= nph;
    else if (2 * d < -nph) d += nph;
  }
  return d;
}

// exact trilinear weights of row (R, ang) on the 27 offsets; false if a
// nonzero weight falls outside {-1, 0, 1}^3
__device__ bool sur_targets(const Tables& tb, const Wt<double>& w, int ang, double* y) {
  for (int q = 0; q < 27; ++q) y[q] = 0.0;
  const int j = ang / tb.n_ph, k = ang % tb.n_ph;
  const int jR = tb.n_mu >= 2 ? w.jL + 1 : w.jL;
  const int kR = tb.n_ph >= 2 ? (w.kL + 1) % tb.n_ph : w.kL;
  bool rep = true;
  for (int ie = 0; ie < 2; ++ie) {
    const double we = ie ? w.we : 1.0 - w.we;
    const int de = w.m + ie;
    for (int ij = 0; ij < 2; ++ij) {
      const double wm = ij ? w.wmu : 1.0 - w.wmu;
      const int dm = (ij ? jR : w.jL) - j;
      for (int ik = 0; ik < 2; ++ik) {
        const double wp = ik ? w.wph : 1.0 - w.wph;
        const int dp = phi_offset((ik ? kR : w.kL) - k, tb.n_ph);
        const double c = we * wm * wp;
        if (c == 0.0) continue;
        if (de < -1 || de > 1 || dm < -1 || dm > 1 || dp < -1 || dp > 1) { rep = false; continue; }
        y[9 * (de + 1) + 3 * (dm + 1) + (dp + 1)] += c;
      }
    }
  }
  if (!rep)
    for (int q = 0; q < 27; ++q) y[q] = 0.0;
  return rep;
}

__global__ void k_sur_samples(Tables tb, State st, const int* idx, long long n, float* X, float* Y, int* valid) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int zone = idx[3 * i], kind = idx[3 * i + 1], ang = idx[3 * i + 2];
    double f[16], y[27];
    for (int q = 0; q < 16; ++q) f[q] = 0.0;
    for (int q = 0; q < 27; ++q) y[q] = 0.0;
    int v = 0;
    FaceDesc F;
    RemapRow R;
    if (zone >= 0 && zone < tb.n_zone && kind >= 0 && kind < kSurKindsAll && ang >= 0 && ang < tb.n_ang &&
        sur_row(tb, st, zone, kind, F, R)) {
      sur_features(tb, R, ang, f);
      Loc<double> LX, LY;
      make_loc(LX, R.vX, R.alX, R.cfX);
      make_loc(LY, R.vY, R.alY, R.cfY);
      const double n3[3] = {f[0], f[1], f[2]};
      Wt<double> w;
      chain_weights_dir<double>(tb, tb.mu, n3, LX, LY, R.G, R.gT, R.axis, make_ebr<double>(tb.R), w);
      v = sur_targets(tb, w, ang, y) ? 1 : 2;
    }
    for (int q = 0; q < 16; ++q) X[16 * i + q] = (float)f[q];
    for (int q = 0; q < 27; ++q) Y[27 * i + q] = (float)y[q];
    valid[i] = v;
  }
}

// ---------------------------------------------------------------------------
// Learned remap in the step: one CTA (one warpgroup) per zone at a time
// evaluates the network on the zone's 31 x n_ang remap rows (tensor cores,
// 128-row tiles), projects each predicted distribution onto the trilinear
// family by its mean offset per axis (exact when the prediction equals the
// exact weights, which are trilinear), and checks it against the exact
// float32 weights of the same row: a row whose mean offsets differ by tol or
// more on any axis trips and takes the exact weights.  Both weight forms sum
// to one per axis, so number is conserved either way.
// ---------------------------------------------------------------------------
struct SurXfer {
  Loc<float> X, Y;
  float G[9];
  float feat[13];   // features 3..15 of every row of this remap
  int hasG, gT, axis, ok;
};

constexpr int kSurT = 128;
constexpr size_t kSurW = (tc::kMlpWBytes + 127) & ~size_t(127);
constexpr size_t kSurX = kSurW;
constexpr size_t kSurH = kSurX + 4096;
constexpr size_t kSurXf = kSurH + 16384;
constexpr size_t kSurDir = kSurXf + ((sizeof(SurXfer) * kSurKindsAll + 127) & ~size_t(127));
constexpr size_t kSurBar = kSurDir + 4 * (3 * kMaxAng + kMaxMu);
constexpr size_t kSurKl = kSurBar + 64;          // the zone's remap kinds to evaluate [32] + count
constexpr size_t kSurBytes = kSurKl + 4 * 33;

__device__ __forceinline__ float mean_offset(const float* p, int axis) {
  // sum over the 27 entries of offset * weight along one axis
  float s = 0.0f;
  for (int q = 0; q < 27; ++q) {
    const int d = axis == 0 ? q / 9 : (axis == 1 ? (q / 3) % 3 : q % 3);
    if (d == 0) s -= p[q];
    else if (d == 2) s += p[q];
  }
  return s;
}

__global__ void __launch_bounds__(kSurT) k_sur_table(Tables tb, State st, const float* __restrict__ prm, float tol,
                                                     int with_time, int split, Wt<float>* __restrict__ tab,
                                                     unsigned long long* counts) {
  extern __shared__ __align__(128) unsigned char smem[];
  const tc::MlpW w = tc::carve_w(smem);
  unsigned char* Xs = smem + kSurX;
  unsigned char* Hs = smem + kSurH;
  SurXfer* xf = reinterpret_cast<SurXfer*>(smem + kSurXf);
  float* n0 = reinterpret_cast<float*>(smem + kSurDir);
  float* n1 = n0 + kMaxAng;
  float* n2 = n1 + kMaxAng;
  float* smu = n2 + kMaxAng;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + kSurBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + kSurBar + 8);
  int* klist = reinterpret_cast<int*>(smem + kSurKl);
  const int t = threadIdx.x;
  const int NA = tb.n_ang, NPH = tb.n_ph, NMU = tb.n_mu;
  tc::stage_w(w, prm);
  for (int q = t; q < NA; q += kSurT) {
    const int j = q / NPH, k = q % NPH;
    n0[q] = (float)tb.mu[j];
    n1[q] = (float)(tb.smu[j] * tb.cph[k]);
    n2[q] = (float)(tb.smu[j] * tb.sph[k]);
  }
  for (int q = t; q < NMU; q += kSurT) smu[q] = (float)tb.mu[q];
  if (t == 0) tc::bar_init(bar);
  if (t < 32) tc::tmem_alloc(slot, 64);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *slot;
  unsigned phase = 0;
  bool ok = true;
  unsigned long long n_eval = 0, n_trip = 0;
  const EBr<float> Rf = make_ebr<float>((float)tb.R);
  for (int zone = blockIdx.x; zone < tb.n_zone && ok; zone += gridDim.x) {
    if (t < kSurKindsAll) {
      SurXfer& x = xf[t];
      FaceDesc F;
      RemapRow R;
      // rows the step reads: the time remap if pending; in the split form
      // only the faces this zone owns (their other side reads them too)
      const bool used = t == 0 ? with_time != 0 : (!split || face_owned(tb, zone % tb.n_r, (t - 1) / 6));
      x.ok = used && sur_row(tb, st, zone, t, F, R);
      if (x.ok) {
        double f[16];
        sur_features(tb, R, 0, f);
        for (int q = 0; q < 13; ++q) x.feat[q] = (float)f[3 + q];
        make_loc(x.X, R.vX, R.alX, R.cfX);
        make_loc(x.Y, R.vY, R.alY, R.cfY);
        x.hasG = R.G != nullptr;
        for (int q = 0; q < 9; ++q) x.G[q] = R.G ? (float)R.G[q] : 0.0f;
        x.gT = R.gT;
        x.axis = R.axis;
      }
    }
    __syncthreads();
    if (t == 0) {   // compact list of the remaps that exist and are used
      int nk = 0;
      for (int k = 0; k < kSurKindsAll; ++k)
        if (xf[k].ok) klist[nk++] = k;
      klist[32] = nk;
    }
    __syncthreads();
    const int rows = klist[32] * NA;
    for (int base = 0; base < rows && ok; base += kSurT) {
      const int q = base + t;
      const bool valid = q < rows;
      const int kind = valid ? klist[q / NA] : 0, ang = q % NA;
      float x[16], z[32], p[27];
      if (valid) {
        const SurXfer& X = xf[kind];
        x[0] = n0[ang]; x[1] = n1[ang]; x[2] = n2[ang];
#pragma unroll
        for (int i = 0; i < 13; ++i) x[3 + i] = X.feat[i];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = (x[i] - w.mean[i]) * w.scale[i];
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = 0.0f;
      }
      ok = tc::tile_forward(w, Xs, Hs, tmem, bar, phase, x, z, st.flag);
      if (!ok || !valid) continue;
      tc::softmax27(z, p);
      const SurXfer& X = xf[kind];
      // exact weights of the row (the check and the fallback)
      Wt<float> ex;
      const float nd[3] = {n0[ang], n1[ang], n2[ang]};
      chain_weights_dir<float>(tb, smu, nd, X.X, X.Y, X.hasG ? X.G : nullptr, X.gT, X.axis, Rf, ex);
      const int j = ang / NPH, k = ang % NPH;
      const float ee = (float)ex.m + ex.we;
      const float em = (float)(ex.jL - j) + ex.wmu;
      const float ep = (float)phi_offset(ex.kL - k, NPH) + ex.wph;
      const float de = mean_offset(p, 0), dm = mean_offset(p, 1), dp = mean_offset(p, 2);
      Wt<float> out = ex;
      const bool trip = !(fabsf(de - ee) < tol && fabsf(dm - em) < tol && fabsf(dp - ep) < tol);
      if (!trip) {
        const float fe = floorf(de), fm = floorf(dm), fp = floorf(dp);
        out.m = (short)fe;
        out.we = de - fe;
        int jl = j + (int)fm;
        float wm = dm - fm;
        if (NMU == 1) { jl = 0; wm = 0.0f; }
        else if (jl < 0) { jl = 0; wm = 0.0f; }
        else if (jl > NMU - 2) { jl = NMU - 2; wm = 1.0f; }
        out.jL = (short)jl;
        out.wmu = wm;
        if (NPH == 1) { out.kL = 0; out.wph = 0.0f; }
        else {
          int kl = (k + (int)fp) % NPH;
          if (kl < 0) kl += NPH;
          out.kL = (short)kl;
          out.wph = dp - fp;
        }
        out.pad = 0;
      }
      tab[((size_t)zone * kSurKindsAll + kind) * NA + ang] = out;
      ++n_eval;
      n_trip += trip ? 1 : 0;
    }
    __syncthreads();
  }
  if (!ok && t == 0) tc::bar_wait(bar, phase ^ 1u, nullptr);
  for (int o = 16; o > 0; o >>= 1) {
    n_eval += __shfl_xor_sync(0xffffffffu, n_eval, o);
    n_trip += __shfl_xor_sync(0xffffffffu, n_trip, o);
  }
  if ((t & 31) == 0) {
    atomicAdd(counts, n_eval);
    atomicAdd(counts + 1, n_trip);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (t < 32) tc::tmem_dealloc(tmem, 64);
}

template <typename T, int NT>
int launch_flux_t(const Tables& tb, const State& st, double dt, cudaStream_t s) {
  size_t sm = flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, NT / 32, 0, default_rb(NT), nullptr, nullptr);
  k_flux_collide<T, NT><<<tb.n_zone, NT, sm, s>>>(tb, st, dt);
  return (int)cudaGetLastError();
}

// split form: the face pass, then the zone pass (both one CTA per zone)
// rows per angular-list walk of the float32 face pass: each thread's rows
// (rows = groups / (threads / angles), rounded up) in as few walks as
// possible without rows masked off -- five rows a walk where the count is a
// multiple of five (20 groups on 128 angles: two walks instead of three),
// two where a thread has at most two.  (Whole blocks also keep the chunk
// layout's padding, and so the shared memory, small.)
template <typename T, int NT>
int face_rb(const Tables& tb) {
  const int nch = chunk_nch(tb.n_ang, NT);
  const int rows = (tb.n_e + nch - 1) / nch;
  if (NT == 384) {
    // the 384-thread face pass (float32 only): seven rows a walk on 20
    // groups x 128 angles (three chunks), else blocks of four
    return (tb.n_e == 20 && tb.n_ang == 128 && tb.n_mu == 16 && tb.n_ph == 8) ? 7 : 4;
  }
  if (rows % 5 == 0) return 5;
  if (sizeof(T) == 4 && NT < 512 && rows <= 2) return 2;
  return default_rb(NT);
}
template <typename T, int NT>
size_t faces_smem(const Tables& tb) {
  return flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, NT / 32, 1, face_rb<T, NT>(tb), nullptr, nullptr);
}
template <typename T, int NT>
int launch_faces_t(const Tables& tb, const State& st, double dt, void* dep, void* rec, cudaStream_t s) {
  const size_t sm1 = faces_smem<T, NT>(tb);
  const int grid = st.zlist ? st.n_zlist : tb.n_zone;
  if (grid <= 0) return 0;
  T* d = reinterpret_cast<T*>(dep);
  DepRec* r = reinterpret_cast<DepRec*>(rec);
  const int rb = face_rb<T, NT>(tb);
  // the benchmark configurations' grids, with the group and angle counts
  // fixed at compile time (constant strides and trip counts); every other
  // problem takes the generic kernel below
  auto grid_is = [&](int ne, int na, int nmu, int nph) {
    return tb.n_e == ne && tb.n_ang == na && tb.n_mu == nmu && tb.n_ph == nph;
  };
  if constexpr (sizeof(T) == 4 && NT == 384) {
    if (rb == 7 && grid_is(20, 128, 16, 8)) {
      k_flux_faces<T, NT, 7, 20, 128, 16, 8><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  if constexpr (sizeof(T) == 4 && NT == 512) {
    if (rb == 5 && grid_is(20, 128, 16, 8)) {
      k_flux_faces<T, NT, 5, 20, 128, 16, 8><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  if constexpr (sizeof(T) == 4 && NT == 256) {
    if (rb == 4 && grid_is(12, 80, 8, 10)) {
      k_flux_faces<T, NT, 4, 12, 80, 8, 10><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
    if (rb == 2 && grid_is(8, 48, 6, 8)) {
      k_flux_faces<T, NT, 2, 8, 48, 6, 8><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  if constexpr (NT != 384) {
    if (rb == 5) {
      k_flux_faces<T, NT, 5><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  if constexpr (sizeof(T) == 4 && NT == 256) {
    if (rb == 2) {
      k_flux_faces<T, NT, 2><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  k_flux_faces<T, NT><<<grid, NT, sm1, s>>>(tb, st, dt, d, r);
  return (int)cudaGetLastError();
}
template <typename T>
int launch_zone_t(const Tables& tb, const State& st, double dt, void* dep, void* rec, cudaStream_t s) {
  size_t sm2 = flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, 256 / 32, 2, default_rb(256), nullptr, nullptr);
  const int grid = st.zlist ? st.n_zlist : tb.n_zone;
  if (grid <= 0) return 0;
  T* d = reinterpret_cast<T*>(dep);
  DepRec* r = reinterpret_cast<DepRec*>(rec);
  if constexpr (sizeof(T) == 4) {
    // the benchmark configurations' grids at compile time (as the face pass)
    auto grid_is = [&](int ne, int na, int nmu, int nph) {
      return tb.n_e == ne && tb.n_ang == na && tb.n_mu == nmu && tb.n_ph == nph;
    };
    if (grid_is(20, 128, 16, 8)) {
      k_zone_collide<T, 20, 128, 16, 8><<<grid, 256, sm2, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
    if (grid_is(12, 80, 8, 10)) {
      k_zone_collide<T, 12, 80, 8, 10><<<grid, 256, sm2, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
    if (grid_is(8, 48, 6, 8)) {
      k_zone_collide<T, 8, 48, 6, 8><<<grid, 256, sm2, s>>>(tb, st, dt, d, r);
      return (int)cudaGetLastError();
    }
  }
  k_zone_collide<T><<<grid, 256, sm2, s>>>(tb, st, dt, d, r);
  return (int)cudaGetLastError();
}

template <typename T, int NT>
int flux_occupancy_t(const Tables& tb) {
  size_t sm = flux_smem_layout<T>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, NT / 32, 0, default_rb(NT), nullptr, nullptr);
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_flux_collide<T, NT>, NT, sm) != cudaSuccess) return 0;
  return blocks;
}
template <typename T, int NT>
int split_occupancy_t(const Tables& tb) {
  const size_t sm = faces_smem<T, NT>(tb);
  int blocks = 0;   // (every RB variant has the same registers)
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_flux_faces<T, NT>, NT, sm) != cudaSuccess) return 0;
  return blocks;
}

template <typename T>
int launch_remap_t(const Tables& tb, const State& st, cudaStream_t s) {
  // 128 threads per CTA (eight CTAs per SM) while one thread per angle
  // fits, else 256: more zones in flight hide the per-zone barriers
  const size_t sm128 = remap_smem_layout<T>(tb.n_e, tb.n_ang, tb.n_mu, 128, nullptr, nullptr);
  if constexpr (sizeof(T) == 4) {
    // the benchmark configurations' grids at compile time (as the face pass)
    auto grid_is = [&](int ne, int na, int nmu, int nph) {
      return tb.n_e == ne && tb.n_ang == na && tb.n_mu == nmu && tb.n_ph == nph;
    };
    if (grid_is(20, 128, 16, 8)) {
      k_time_remap<T, 128, 20, 128, 16, 8><<<tb.n_zone, 128, sm128, s>>>(tb, st);
      return (int)cudaGetLastError();
    }
    if (grid_is(12, 80, 8, 10)) {
      k_time_remap<T, 128, 12, 80, 8, 10><<<tb.n_zone, 128, sm128, s>>>(tb, st);
      return (int)cudaGetLastError();
    }
    if (grid_is(8, 48, 6, 8)) {
      k_time_remap<T, 128, 8, 48, 6, 8><<<tb.n_zone, 128, sm128, s>>>(tb, st);
      return (int)cudaGetLastError();
    }
  }
  if (tb.n_ang <= 128)
    k_time_remap<T, 128><<<tb.n_zone, 128, sm128, s>>>(tb, st);
  else
    k_time_remap<T, 256><<<tb.n_zone, 256, remap_smem_layout<T>(tb.n_e, tb.n_ang, tb.n_mu, 256, nullptr, nullptr), s>>>(
        tb, st);
  return (int)cudaGetLastError();
}

}  // namespace

size_t flux_smem_bytes(const Tables& tb, int mixed, int nt) {
  const int threads = nt & 0xFFFF;
  if (nt & kShapeSplit) {
    size_t a = threads >= 512   ? (mixed ? faces_smem<float, 512>(tb) : faces_smem<double, 512>(tb))
               : threads == 384 ? faces_smem<float, 384>(tb)   // (float32 only; not offered in float64)
                                : (mixed ? faces_smem<float, 256>(tb) : faces_smem<double, 256>(tb));
    size_t b = mixed ? flux_smem_layout<float>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, 8, 2, 4, nullptr, nullptr)
                     : flux_smem_layout<double>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, 8, 2, 4, nullptr, nullptr);
    return a > b ? a : b;
  }
  return mixed ? flux_smem_layout<float>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, threads / 32, 0, default_rb(threads), nullptr,
                                         nullptr)
               : flux_smem_layout<double>(tb.n_s, tb.n_e, tb.n_ang, tb.n_mu, threads / 32, 0, default_rb(threads), nullptr,
                                          nullptr);
}
size_t split_dep_bytes(const Tables& tb, int mixed) {
  return (size_t)tb.n_zone * 6 * tb.n_s * tb.n_e * tb.n_ang * (mixed ? 4 : 8);
}
size_t split_rec_bytes(const Tables& tb) { return (size_t)tb.n_zone * 6 * tb.n_s * sizeof(DepRec); }
size_t remap_smem_bytes(const Tables& tb, int mixed) {
  const int nt = tb.n_ang <= 128 ? 128 : 256;   // the launch's shape (launch_remap_t)
  return mixed ? remap_smem_layout<float>(tb.n_e, tb.n_ang, tb.n_mu, nt, nullptr, nullptr)
               : remap_smem_layout<double>(tb.n_e, tb.n_ang, tb.n_mu, nt, nullptr, nullptr);
}
// Allow the large dynamic shared-memory carve-outs once (a function
// attribute, set outside any stream capture).
int prepare_kernels() {
  int dev = 0, lim = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaError_t e = cudaSuccess;
#define BT_SET(fn) if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
  BT_SET((k_flux_collide<float, 128>));
  BT_SET((k_flux_collide<float, 256>));
  BT_SET((k_flux_collide<float, 512>));
  BT_SET((k_flux_collide<double, 128>));
  BT_SET((k_flux_collide<double, 256>));
  BT_SET((k_flux_collide<double, 512>));
  BT_SET((k_flux_faces<float, 256>));
  BT_SET((k_flux_faces<float, 256, 5>));
  BT_SET((k_flux_faces<float, 256, 2>));
  BT_SET((k_flux_faces<float, 512>));
  BT_SET((k_flux_faces<float, 512, 5>));
  BT_SET((k_flux_faces<float, 512, 5, 20, 128, 16, 8>));
  BT_SET((k_flux_faces<float, 384>));
  BT_SET((k_flux_faces<float, 384, 7, 20, 128, 16, 8>));
  BT_SET((k_flux_faces<float, 256, 4, 12, 80, 8, 10>));
  BT_SET((k_flux_faces<float, 256, 2, 8, 48, 6, 8>));
  BT_SET((k_flux_faces<double, 256>));
  BT_SET((k_flux_faces<double, 256, 5>));
  BT_SET((k_flux_faces<double, 512>));
  BT_SET((k_flux_faces<double, 512, 5>));
  BT_SET((k_zone_collide<float>));
  BT_SET((k_zone_collide<float, 12, 80, 8, 10>));
  BT_SET((k_zone_collide<float, 20, 128, 16, 8>));
  BT_SET((k_zone_collide<float, 8, 48, 6, 8>));
  BT_SET((k_zone_collide<double>));
  BT_SET((k_time_remap<float, 128>));
  BT_SET((k_time_remap<float, 128, 20, 128, 16, 8>));
  BT_SET((k_time_remap<float, 128, 12, 80, 8, 10>));
  BT_SET((k_time_remap<float, 128, 8, 48, 6, 8>));
  BT_SET((k_time_remap<float, 256>));
  BT_SET((k_time_remap<double, 128>));
  BT_SET((k_time_remap<double, 256>));
  BT_SET(k_sur_table);
#undef BT_SET
  return (int)e;
}

int flux_occupancy(const Tables& tb, int mixed, int nt) {
  if (nt & kShapeSplit) {
    switch (nt & 0xFFFF) {
      case 256: return mixed ? split_occupancy_t<float, 256>(tb) : split_occupancy_t<double, 256>(tb);
      case 512: return mixed ? split_occupancy_t<float, 512>(tb) : split_occupancy_t<double, 512>(tb);
      case 384: return mixed ? split_occupancy_t<float, 384>(tb) : 0;   // float32 only
      default: return 0;
    }
  }
  switch (nt) {
    case 128: return mixed ? flux_occupancy_t<float, 128>(tb) : flux_occupancy_t<double, 128>(tb);
    case 512: return mixed ? flux_occupancy_t<float, 512>(tb) : flux_occupancy_t<double, 512>(tb);
    default: return mixed ? flux_occupancy_t<float, 256>(tb) : flux_occupancy_t<double, 256>(tb);
  }
}

int max_optin_smem() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

int launch_flux_collide(const Tables& tb, const State& st, double dt, int mixed, int nt, void* dep, void* rec,
                        void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (nt & kShapeSplit) {
    if (!dep || !rec) return (int)cudaErrorInvalidValue;
    if ((nt & 0xFFFF) == 512)
      return mixed ? launch_faces_t<float, 512>(tb, st, dt, dep, rec, s) : launch_faces_t<double, 512>(tb, st, dt, dep, rec, s);
    if ((nt & 0xFFFF) == 384)
      return mixed ? launch_faces_t<float, 384>(tb, st, dt, dep, rec, s) : (int)cudaErrorInvalidValue;
    return mixed ? launch_faces_t<float, 256>(tb, st, dt, dep, rec, s) : launch_faces_t<double, 256>(tb, st, dt, dep, rec, s);
  }
  switch (nt) {
    case 128: return mixed ? launch_flux_t<float, 128>(tb, st, dt, s) : launch_flux_t<double, 128>(tb, st, dt, s);
    case 512: return mixed ? launch_flux_t<float, 512>(tb, st, dt, s) : launch_flux_t<double, 512>(tb, st, dt, s);
    default: return mixed ? launch_flux_t<float, 256>(tb, st, dt, s) : launch_flux_t<double, 256>(tb, st, dt, s);
  }
}

int launch_zone_collide(const Tables& tb, const State& st, double dt, int mixed, void* dep, void* rec, void* stream) {
  if (!dep || !rec) return (int)cudaErrorInvalidValue;
  cudaStream_t s = (cudaStream_t)stream;
  return mixed ? launch_zone_t<float>(tb, st, dt, dep, rec, s) : launch_zone_t<double>(tb, st, dt, dep, rec, s);
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

int launch_max_rate(const Tables& tb, const State& st, double* d_rate, void* stream, double* d_zone_rates) {
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(d_rate, 0, sizeof(double), s);
  k_max_rate<<<tb.n_zone, kThreads, 0, s>>>(tb, st, reinterpret_cast<unsigned long long*>(d_rate), d_zone_rates);
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

size_t sur_table_bytes(const Tables& tb) { return sizeof(Wt<float>) * (size_t)tb.n_zone * kSurKindsAll * tb.n_ang; }

int launch_sur_table(const Tables& tb, const State& st, const float* prm, float tol, int with_time, int split,
                     void* tab, unsigned long long* counts, int grid, void* stream) {
  const int g = grid < tb.n_zone ? grid : tb.n_zone;
  k_sur_table<<<g, kSurT, kSurBytes, (cudaStream_t)stream>>>(tb, st, prm, tol, with_time, split,
                                                             reinterpret_cast<Wt<float>*>(tab), counts);
  return (int)cudaGetLastError();
}

int launch_sur_samples(const Tables& tb, const State& st, const int* idx, long long n, float* X, float* Y, int* valid,
                       void* stream) {
  if (n <= 0) return 0;
  long long blocks = (n + 127) / 128;
  if (blocks > 8192) blocks = 8192;
  k_sur_samples<<<(int)blocks, 128, 0, (cudaStream_t)stream>>>(tb, st, idx, n, X, Y, valid);
  return (int)cudaGetLastError();
}

}  // namespace bt
