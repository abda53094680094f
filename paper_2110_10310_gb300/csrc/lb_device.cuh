#pragma once

// Device code shared by the kernel translation units of the implicit-midpoint
// Lindblad path (sm_103a, FP64): reductions, the predictor weights, the
// problem header copied into shared memory and the matrix-free off-diagonal
// apply.  Everything is in an unnamed namespace: each translation unit
// gets its own copy.
//
//
// Design notes
// * The vectorised Lindbladian M(t) of Appendix A (eq. mastereq_vectorized)
//   is never formed.  For vec index v = k + N l (column stacking) it acts as
//     (M x)_kl = D_kl x_kl + sum_q [ jump_q + control_q ](k, l)
//   where D is diagonal and time independent (Hamiltonian diagonal, all
//   anticommutator terms and the dephasing sandwich L_2q x L_2q), the jump
//   term couples x_{k+s_q, l+s_q} (decay sandwich L_1q x L_1q) and the
//   control term couples x_{k+-s_q, l} and x_{k, l-+s_q} (-i[H_c, x]), s_q
//   being the index stride of subsystem q.
// * FP64 is the binding resource on this GPU (two FP64 lanes per SM per
//   clock, one warp instruction per 64 cycles per SM sub-partition, whatever
//   the number of active lanes), so the kernels minimise FP64 instructions:
//   coefficient selection and index arithmetic run on the integer pipe, and
//   per-element coefficients come from small tables.
// * Inner solve of (I - dt/2 M) z = q (eq. linsystem_primal): Jacobi
//   fixed point z <- (I - dt/2 D)^-1 (q + dt/2 O z), O = M - D, from
//   z_0 = (I - dt/2 D)^-1 q, to ||z_new - z||_inf <= rtol ||q||_inf.  The
//   maximum is taken on the integer bit patterns of |.|, so the stopping
//   decision is exact and identical in a recompute.
// * "Resident" kernels: one CTA owns one state (V = N^2 <= 4096) in shared
//   memory and runs the whole time loop; the CTA barrier is the only
//   synchronisation of an inner iteration.

#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "lb_internal.h"

namespace cg = cooperative_groups;

namespace lbk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ULL;
constexpr double kTwoPi = 6.283185307179586476925286766559;

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = umax64(x, __shfl_xor_sync(kFull, x, o));
  return x;
}
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}
// Sum of four per-lane values over the warp with 6 FP64 additions per lane:
// after the call lane 0 holds the total of v0, lane 8 of v1, lane 16 of v2 and
// lane 24 of v3.
__device__ __forceinline__ double warp_sum4(double v0, double v1, double v2, double v3, int lane) {
  const bool h16 = lane & 16;
  double k0 = h16 ? v2 : v0, k1 = h16 ? v3 : v1;
  const double s0 = h16 ? v0 : v2, s1 = h16 ? v1 : v3;
  k0 += __shfl_xor_sync(kFull, s0, 16);
  k1 += __shfl_xor_sync(kFull, s1, 16);
  const bool h8 = lane & 8;
  double k = h8 ? k1 : k0;
  const double s = h8 ? k0 : k1;
  k += __shfl_xor_sync(kFull, s, 8);
  k += __shfl_xor_sync(kFull, k, 4);
  k += __shfl_xor_sync(kFull, k, 2);
  k += __shfl_xor_sync(kFull, k, 1);
  return k;
}

// Sum of two per-lane values over the warp with 5 FP64 additions per lane:
// after the call lane 0 holds the total of a and lane 16 that of b.
__device__ __forceinline__ double warp_sum2(double a, double b, int lane) {
  const bool h16 = lane & 16;
  double k = h16 ? b : a;
  k += __shfl_xor_sync(kFull, h16 ? a : b, 16);
  k += __shfl_xor_sync(kFull, k, 8);
  k += __shfl_xor_sync(kFull, k, 4);
  k += __shfl_xor_sync(kFull, k, 2);
  k += __shfl_xor_sync(kFull, k, 1);
  return k;
}

// First-iterate predictor of every sweep: the off-diagonal correction
// c_j = (I - dt/2 D) z^j - rhs^j of a step is extrapolated by the polynomial
// through the last n recorded ones, c_j ~ sum_{i=1..n} (-1)^(i+1) binom(n, i)
// c_{j-i}, n <= kPredOrder; the table holds these weights for each n.
static_assert(kPredOrder == 7, "the weight table below is written for order 7");
__constant__ double kExtrap[kPredOrder + 1][kPredOrder] = {
    {0, 0, 0, 0, 0, 0, 0},         {1, 0, 0, 0, 0, 0, 0},          {2, -1, 0, 0, 0, 0, 0},
    {3, -3, 1, 0, 0, 0, 0},        {4, -6, 4, -1, 0, 0, 0},        {5, -10, 10, -5, 1, 0, 0},
    {6, -15, 20, -15, 6, -1, 0},   {7, -21, 35, -35, 21, -7, 1}};

// The grid and one-CTA sweeps extrapolate in the frame that follows each
// element's own free evolution.  One implicit-midpoint step of the diagonal
// part alone multiplies element v by g_v = (1 + dt/2 D_v)/(1 - dt/2 D_v)
// = 2 (1 - dt/2 D_v)^-1 - 1 (its complex conjugate for the adjoint), so the
// corrections c_{j-i} g_v^i of the previous steps carry only the slow
// remainder of the motion, and the prediction is
//   c_j ~ sum_{i=1..n} (-1)^(i+1) binom(n, i) g_v^i c_{j-i},  n <= kRingOrder.
// Without the rotation the fast diagonal phases (h |E_k - E_l| up to a few
// tenths of a radian per step on the six-qutrit system) limit the order-7
// extrapolation to a first iterate several digits short of the tolerance.
// The corrections are recorded as computed by the last inner iteration (the
// off-diagonal sum alone, accurate relative to |c|), not as
// (I - dt/2 D) z - rhs, whose cancellation leaves rounding errors of order
// eps |q| that the weights (their magnitudes sum to 2^n - 1) would amplify
// to the size of the stopping tolerance.
static_assert(kRingOrder == 10, "the weight table below is written for order 10");
__constant__ double kExtrapR[kRingOrder + 1][kRingOrder] = {
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {1, 0, 0, 0, 0, 0, 0, 0, 0, 0},
    {2, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {3, -3, 1, 0, 0, 0, 0, 0, 0, 0},
    {4, -6, 4, -1, 0, 0, 0, 0, 0, 0},
    {5, -10, 10, -5, 1, 0, 0, 0, 0, 0},
    {6, -15, 20, -15, 6, -1, 0, 0, 0, 0},
    {7, -21, 35, -35, 21, -7, 1, 0, 0, 0},
    {8, -28, 56, -70, 56, -28, 8, -1, 0, 0},
    {9, -36, 84, -126, 126, -84, 36, -9, 1, 0},
    {10, -45, 120, -210, 252, -210, 120, -45, 10, -1}};

// The ring holds the corrections in the frame of an anchor step,
// c~_j = g^-m_j c_j with m_j the steps since the anchor and g the element's
// free step factor, so that the prediction
//   c_j ~ sum_{i=1..n} w_i g^i c_{j-i} = g^m_j sum_i w_i c~_{j-i}
// costs one weighted sum of the ring (integer weights, on the integer pipe:
// wsum_int) and one complex product; the powers g^m and g^-m are kept per
// element and advanced once per step.  The anchor is the last restart, or
// moves every kAnchorSteps steps (the ring's entries are then brought to the
// new frame), so that the powers stay within a few hundred factors of
// rounding.
constexpr int kAnchorSteps = 256;

// The extrapolation weights as integers, kExtrapR[n][k-1] = (-1)^(k+1) C(n, k)
__host__ __device__ constexpr int extrap_weight(int n, int k) {
  int c = 1;
  for (int j = 1; j <= k; ++j) c = c * (n - j + 1) / j;
  return (k & 1) ? c : -c;
}
__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double dfrom(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ int clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}

// sum_i w_i x_i of NC doubles with the integer weights of the order-NC
// extrapolation (x_0 the oldest), on the integer pipe (the FP64 pipe bounds
// the sweeps): every x_i as its 53-bit significand aligned to the largest
// exponent (the bits below the alignment truncated), the weighted sum exact
// in 64 bits (|w_i| <= 252 and sum |w_i| < 2^10, so |sum| < 2^63), then
// truncated to double.  The error is below sum |w_i| 2^-52 max |x_i|, the
// size of an FP64 multiply-add chain's; sums below the normal range are
// flushed to zero, and a non-finite x_i gives NaN.
template <int NC>
__host__ __device__ __forceinline__ double wsum_int(const double (&x)[NC]) {
  unsigned long long b[NC];
  int emax = 1;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    b[i] = dbits(x[i]);
    const int e = (int)(b[i] >> 52) & 0x7ff;
    emax = e > emax ? e : emax;
  }
  if (emax == 0x7ff) return dfrom(0x7ff8000000000000ull);
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const int e = (int)(b[i] >> 52) & 0x7ff;
    const unsigned long long m = (b[i] & 0xfffffffffffffull) | (e ? 0x10000000000000ull : 0ull);
    const int sh = emax - (e ? e : 1);  // a subnormal has the scale of exponent field 1
    const long long t = sh < 53 ? (long long)(m >> sh) : 0ll;
    const int w = extrap_weight(NC, NC - i);
    acc += (long long)((b[i] >> 63) ? -w : w) * t;
  }
  if (acc == 0) return 0.0;
  const unsigned long long sg = acc < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = acc < 0 ? 0ull - (unsigned long long)acc : (unsigned long long)acc;
  const int lz = clz64(a);
  a <<= lz;                     // leading bit at 63: the sum is a 2^(emax - 1075 - lz)
  const int E = emax + 11 - lz;  // its biased exponent
  if (E <= 0) return dfrom(sg);
  if (E >= 0x7ff) return dfrom(sg | 0x7ff0000000000000ull);
  return dfrom(sg | ((unsigned long long)E << 52) | ((a >> 11) & 0xfffffffffffffull));
}

// sum_{i=1..n} w_i c~_{j-i} of one element (real weights, the ring in the
// anchor frame); NO: n as a compile-time constant (the sum on the integer
// pipe), 0 = runtime n (the warm-up steps after a restart, in FP64)
template <int NO>
__device__ __forceinline__ double2 anchored_sum_n(const double2* __restrict__ ring, size_t stride, int slot, int n) {
  constexpr int NC = NO > 0 ? NO : 1;
  if (NO > 0) n = NO;
  int sl = slot - n;
  if (sl < 0) sl += kRingOrder;
  double pr = 0.0, pi = 0.0;
  if constexpr (NO > 0) {
    double cr[NC], ci[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int s = sl + i < kRingOrder ? sl + i : sl + i - kRingOrder;
      const double2 c = ring[(size_t)s * stride];
      cr[i] = c.x;
      ci[i] = c.y;
    }
    pr = wsum_int<NC>(cr);
    pi = wsum_int<NC>(ci);
  } else {
    for (int i = n; i >= 1; --i) {
      const double2 c = ring[(size_t)sl * stride];
      const double w = kExtrapR[n][i - 1];
      pr = fma(w, c.x, pr);
      pi = fma(w, c.y, pi);
      sl = sl + 1 < kRingOrder ? sl + 1 : 0;
    }
  }
  return make_double2(pr, pi);
}
__device__ __forceinline__ double2 anchored_sum(const double2* __restrict__ ring, size_t stride, int slot, int n) {
  switch (n) {
    case 8: return anchored_sum_n<8>(ring, stride, slot, n);
    case 9: return anchored_sum_n<9>(ring, stride, slot, n);
    case 10: return anchored_sum_n<10>(ring, stride, slot, n);
    default: return anchored_sum_n<0>(ring, stride, slot, n);
  }
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}


// quadratic B-spline of unit knot spacing centred at 0 (Sec. II, eq. rotctrl)
__device__ __forceinline__ double bspline2(double x) {
  x = fabs(x);
  if (x < 0.5) return 0.75 - x * x;
  if (x < 1.5) {
    const double y = x - 1.5;
    return 0.5 * y * y;
  }
  return 0.0;
}

// J from the sum the kernels reduce: 1/2 sum |q - t|^2 for J_Frob, else
// sum Re(conj(t) q): J_Tr = 1 - Re Tr(t^+ q), J_Nm = Re Tr(N_m q) (t = N_m)
// (Sec. III, eq. Jmeasure)
__device__ __forceinline__ double merit_value(int kind, double sum) {
  return kind == LB_J_FROB ? 0.5 * sum : (kind == LB_J_TR ? 1.0 - sum : sum);
}
// factor of the target in the terminal condition beta_i/M g_i for the
// functionals linear in q: g = -t (J_Tr), g = N_m = t (J_Nm)
__device__ __forceinline__ double linear_sign(int kind) { return kind == LB_J_NM ? 1.0 : -1.0; }

__device__ void record_error(DevStatus* st, int code, int step) {
  if (atomicCAS(&st->code, 0, code) == 0) st->step = step;
}

// Factor of the stopping test of step j.  The Jacobi iteration matrix
// T_j = (I - dt/2 D)^-1 dt/2 O_j (and its adjoint) has infinity norm at most
// rho_j (k_stop_factors); when rho_j < 1/2, ||z - z*|| <= rho_j/(1 - rho_j)
// ||z_new - z||, so the test ||z_new - z|| < rtol ||q|| (1 - rho_j)/rho_j
// bounds the error of the returned iterate by rtol ||q||.  Otherwise (and for
// the Neumann iteration) the factor is 1: the plain increment test.
__device__ __forceinline__ double stop_factor(const ProbDev& P, int j) {
  return P.method == LB_SOLVER_JACOBI ? P.sfac[j] : 1.0;
}

// ---------------------------------------------------------------------------
// per-CTA copy of the problem constants used in the inner loops

struct Hdr {
  int Q, N, V, NT, K, n_ckpt, max_iter, method, kind, M, krylov;
  int db, dm;  // bits per packed digit and their mask
  int npair, cq;  // Jaynes-Cummings pairs, entries per step of the control table
  double gamma1;  // weight of the running penalty (0: none)
  int herm, Vh;   // Hermitian symmetry: only the Vh = N (N + 1) / 2 elements k <= l are iterated
  int jp[LB_MAXQ * (LB_MAXQ - 1) / 2], jq[LB_MAXQ * (LB_MAXQ - 1) / 2];
  double h, rtol;
  int lev[LB_MAXQ], stride[LB_MAXQ], coff[LB_MAXQ], joff[LB_MAXQ];
  double jump[LB_MAXQ];
  unsigned jon;  // bit q set when subsystem q decays (jump[q] != 0), tested on the integer pipe
};

struct Tabs {
  const double* cu;
  const double* cd;
  const double* jf;
  const double* ja;
};

__device__ void load_hdr(Hdr& H, const ProbDev& P) {
  H.Q = P.Q;
  H.N = P.N;
  H.V = P.V;
  H.NT = P.NT;
  H.K = P.K;
  H.n_ckpt = P.n_ckpt;
  H.max_iter = P.max_iter;
  H.method = P.method;
  H.kind = P.kind;
  H.M = P.M;
  H.krylov = P.krylov;
  H.db = P.dbits;
  H.dm = (1 << P.dbits) - 1;
  H.npair = P.npair;
  H.cq = P.cq;
  H.gamma1 = P.gamma1;
  H.herm = P.herm;
  H.Vh = P.N * (P.N + 1) / 2;
  for (int k = 0; k < P.npair; ++k) {
    H.jp[k] = P.jp[k];
    H.jq[k] = P.jq[k];
  }
  H.h = P.h;
  H.rtol = P.rtol;
  for (int q = 0; q < LB_MAXQ; ++q) {
    H.lev[q] = P.levels[q];
    H.stride[q] = P.stride[q];
    H.coff[q] = P.coff[q];
    H.joff[q] = P.joff[q];
    H.jump[q] = P.jump[q];
  }
  H.jon = 0u;
  for (int q = 0; q < P.Q; ++q)
    if (P.jump[q] != 0.0) H.jon |= 1u << q;
}

// (dt/2) (O x)_v accumulated into (ar, ai); O = M - D (or its adjoint part
// for ADJ).  x is indexed by the state-local vec index; ct[q] = (dt/2) d_q.
// Load of an iterate element: shared memory / same-CTA data (CG = false), or
// global memory written by other SMs in this launch (CG = true: bypass L1,
// whose lines are not kept coherent across SMs).
template <bool CG>
__device__ __forceinline__ double2 ldz(const double2* p) {
  if constexpr (CG) {
    return __ldcg(p);
  } else {
    return *p;
  }
}

// Entry (k, l) of a Hermitian matrix stored packed, column by column over
// k <= l (entry (k, l) at l (l + 1)/2 + k): entries below the diagonal are the
// conjugates of their mirrors (the sign flip on the integer pipe).
template <bool CG>
__device__ __forceinline__ double2 ldpk(const double2* p, int k, int l) {
  const bool lo = k > l;
  const int a = lo ? l : k, c = lo ? k : l;
  double2 x = ldz<CG>(p + ((c * (c + 1)) >> 1) + a);
  x.y = __longlong_as_double(__double_as_longlong(x.y) ^ (lo ? (long long)0x8000000000000000ULL : 0LL));
  return x;
}

// PK: x is one state stored packed (ldpk), and the neighbours are addressed
// by (k, l) of element v = k + N l; else x is indexed by the vec index.
// QN > 0: H.Q as a compile-time count (the subsystem loop unrolls, so the
// loads and the arithmetic of different subsystems can interleave).
template <bool ADJ, bool CG = false, bool PK = false, int QN = 0>
__device__ __forceinline__ void offdiag_acc(double& ar, double& ai, const double2* __restrict__ x, int v, uint32_t kd,
                                            uint32_t ld, const Hdr& H, const Tabs& T, const double2* __restrict__ ct,
                                            int k = 0, int l = 0) {
  const int N = H.N;
  // entry at row offset dk and column offset dl from the element
  auto nb = [&](int dk, int dl) -> double2 {
    if constexpr (PK) return ldpk<CG>(x, k + dk, l + dl);
    else return ldz<CG>(x + v + dk + dl * N);
  };
  auto sub = [&](int q) {
    const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
    const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
    // control: -i[H_c, X] with H_c = d a + conj(d) a^+ (Sec. II):
    //   P = sqrt(nk+1) x[k+s,l] - sqrt(nl) x[k,l-s]     (a X - X a)
    //   R = sqrt(nk) x[k-s,l] - sqrt(nl+1) x[k,l+s]     (a^+ X - X a^+)
    //   -i d P - i conj(d) R = b (P - R) - i a (P + R), d = (a + i b) * 2/dt
    const double c1 = T.cu[co + nk], c2 = T.cd[co + nl], c3 = T.cd[co + nk], c4 = T.cu[co + nl];
    const double2 x1 = nb(nk + 1 < n ? s : 0, 0);
    const double2 x2 = nb(0, nl > 0 ? -s : 0);
    const double2 x3 = nb(nk > 0 ? -s : 0, 0);
    const double2 x4 = nb(0, nl + 1 < n ? s : 0);
    const double pr = fma(-c2, x2.x, c1 * x1.x);
    const double pi = fma(-c2, x2.y, c1 * x1.y);
    const double rr = fma(-c4, x4.x, c3 * x3.x);
    const double ri = fma(-c4, x4.y, c3 * x3.y);
    const double ur = pr + rr, ui = pi + ri, wr = pr - rr, wi = pi - ri;
    const double2 c = ct[q];
    // the Hamiltonian part of M^+ is minus that of M
    const double a = ADJ ? -c.x : c.x, b = ADJ ? -c.y : c.y;
    ar = fma(b, wr, fma(a, ui, ar));
    ai = fma(b, wi, fma(-a, ur, ai));
    if ((H.jon >> q) & 1u) {
      // decay sandwich: M couples x[k+s, l+s], M^+ couples x[k-s, l-s]
      const int jo = H.joff[q] + nk * n + nl;
      double cj;
      double2 x5;
      if (!ADJ) {
        cj = T.jf[jo];
        const int d = (nk + 1 < n && nl + 1 < n) ? s : 0;
        x5 = nb(d, d);
      } else {
        cj = T.ja[jo];
        const int d = (nk > 0 && nl > 0) ? s : 0;
        x5 = nb(-d, -d);
      }
      ar = fma(cj, x5.x, ar);
      ai = fma(cj, x5.y, ai);
    }
  };
  if constexpr (QN > 0) {
#pragma unroll
    for (int q = 0; q < QN; ++q) sub(q);
  } else {
    for (int q = 0; q < H.Q; ++q) sub(q);
  }
  // Jaynes-Cummings pairs (Sec. II): -i[G a_p^+ a_q + conj(G) a_p a_q^+, X] with
  //   U = sqrt(np_k) sqrt(nq_k+1) x[k-sp+sq, l] - sqrt(np_l+1) sqrt(nq_l) x[k, l+sp-sq]
  //   W = sqrt(np_k+1) sqrt(nq_k) x[k+sp-sq, l] - sqrt(np_l) sqrt(nq_l+1) x[k, l-sp+sq]
  //   -i G U - i conj(G) W = b (U - W) - i a (U + W), (a + i b) = (dt/2) G
  for (int k = 0; k < H.npair; ++k) {
    const int p = H.jp[k], q = H.jq[k];
    const int np = H.lev[p], nq = H.lev[q], sp = H.stride[p], sq = H.stride[q];
    const int pk = (kd >> (H.db * p)) & H.dm, qk = (kd >> (H.db * q)) & H.dm;
    const int pl = (ld >> (H.db * p)) & H.dm, ql = (ld >> (H.db * q)) & H.dm;
    const double u1 = T.cd[H.coff[p] + pk] * T.cu[H.coff[q] + qk];
    const double u2 = T.cu[H.coff[p] + pl] * T.cd[H.coff[q] + ql];
    const double w1 = T.cu[H.coff[p] + pk] * T.cd[H.coff[q] + qk];
    const double w2 = T.cd[H.coff[p] + pl] * T.cu[H.coff[q] + ql];
    const int d = sq - sp;  // row offset of a_p^+ a_q
    const double2 xu1 = nb((pk > 0 && qk + 1 < nq) ? d : 0, 0);
    const double2 xu2 = nb(0, (ql > 0 && pl + 1 < np) ? -d : 0);
    const double2 xw1 = nb((qk > 0 && pk + 1 < np) ? -d : 0, 0);
    const double2 xw2 = nb(0, (pl > 0 && ql + 1 < nq) ? d : 0);
    const double ur = fma(-u2, xu2.x, u1 * xu1.x), ui = fma(-u2, xu2.y, u1 * xu1.y);
    const double wr = fma(-w2, xw2.x, w1 * xw1.x), wi = fma(-w2, xw2.y, w1 * xw1.y);
    const double2 c = ct[H.Q + k];
    const double a = ADJ ? -c.x : c.x, b = ADJ ? -c.y : c.y;
    ar = fma(b, ur - wr, fma(a, ui + wi, ar));
    ai = fma(b, ui - wi, fma(-a, ur + wr, ai));
  }
}


__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__device__ __forceinline__ unsigned hi_abs(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}
constexpr unsigned kInfHi = 0x7ff00000u;

struct CtaStats {
  unsigned long long iters[3] = {0, 0, 0}, steps[3] = {0, 0, 0};
  int maxit = 0;
  __device__ void add(int phase, int it) {
    iters[phase] += it;
    steps[phase] += 1;
    maxit = it > maxit ? it : maxit;
  }
  __device__ void flush(DevStatus* st) {
    if (threadIdx.x == 0) {
      for (int p = 0; p < 3; ++p)
        if (steps[p]) {
          atomicAdd(&st->iters[p], iters[p]);
          atomicAdd(&st->steps[p], steps[p]);
        }
      atomicMax(&st->max_iter_seen, maxit);
    }
  }
};

}  // namespace
}  // namespace lbk
