// CUDA kernels of the implicit-midpoint Lindblad path (sm_103a, FP64).
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

template <bool ADJ, bool CG = false>
__device__ __forceinline__ void offdiag_acc(double& ar, double& ai, const double2* __restrict__ x, int v, uint32_t kd,
                                            uint32_t ld, const Hdr& H, const Tabs& T, const double2* __restrict__ ct) {
  const int N = H.N;
  for (int q = 0; q < H.Q; ++q) {
    const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
    const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
    const int sN = s * N;
    // control: -i[H_c, X] with H_c = d a + conj(d) a^+ (Sec. II):
    //   P = sqrt(nk+1) x[k+s,l] - sqrt(nl) x[k,l-s]     (a X - X a)
    //   R = sqrt(nk) x[k-s,l] - sqrt(nl+1) x[k,l+s]     (a^+ X - X a^+)
    //   -i d P - i conj(d) R = b (P - R) - i a (P + R), d = (a + i b) * 2/dt
    const double c1 = T.cu[co + nk], c2 = T.cd[co + nl], c3 = T.cd[co + nk], c4 = T.cu[co + nl];
    const double2 x1 = ldz<CG>(x + v + (nk + 1 < n ? s : 0));
    const double2 x2 = ldz<CG>(x + v - (nl > 0 ? sN : 0));
    const double2 x3 = ldz<CG>(x + v - (nk > 0 ? s : 0));
    const double2 x4 = ldz<CG>(x + v + (nl + 1 < n ? sN : 0));
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
    if (H.jump[q] != 0.0) {
      // decay sandwich: M couples x[k+s, l+s], M^+ couples x[k-s, l-s]
      const int jo = H.joff[q] + nk * n + nl;
      double cj;
      double2 x5;
      if (!ADJ) {
        cj = T.jf[jo];
        x5 = ldz<CG>(x + v + ((nk + 1 < n && nl + 1 < n) ? s + sN : 0));
      } else {
        cj = T.ja[jo];
        x5 = ldz<CG>(x + v - ((nk > 0 && nl > 0) ? s + sN : 0));
      }
      ar = fma(cj, x5.x, ar);
      ai = fma(cj, x5.y, ai);
    }
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
    const double2 xu1 = ldz<CG>(x + v + ((pk > 0 && qk + 1 < nq) ? d : 0));
    const double2 xu2 = ldz<CG>(x + v - ((ql > 0 && pl + 1 < np) ? d * N : 0));
    const double2 xw1 = ldz<CG>(x + v - ((qk > 0 && pk + 1 < np) ? d : 0));
    const double2 xw2 = ldz<CG>(x + v + ((pl > 0 && ql + 1 < nq) ? d * N : 0));
    const double ur = fma(-u2, xu2.x, u1 * xu1.x), ui = fma(-u2, xu2.y, u1 * xu1.y);
    const double wr = fma(-w2, xw2.x, w1 * xw1.x), wi = fma(-w2, xw2.y, w1 * xw1.y);
    const double2 c = ct[H.Q + k];
    const double a = ADJ ? -c.x : c.x, b = ADJ ? -c.y : c.y;
    ar = fma(b, ur - wr, fma(a, ui + wi, ar));
    ai = fma(b, ui - wi, fma(-a, ur + wr, ai));
  }
}

// ---------------------------------------------------------------------------
// resident kernels: shared-memory layout

struct ResSmem {
  Hdr* hdr;
  double* cu;
  double* cd;
  double* jf;
  double* ja;
  uint32_t* dig;
  uint16_t* hmap;             // [N (N + 1) / 2] vec indices of the elements k <= l (Hermitian symmetry)
  uint16_t* hmir;             // [N (N + 1) / 2] their mirror elements l + N k (0xffff on the diagonal)
  unsigned long long* slots;  // [3][16]
  double* red;                // [4 * LB_MAXQ][16]
  double2* dsm;               // [V] Dinv (Jacobi) or dt/2 D (Neumann)
  double2* zb0;               // [V]
  double2* zb1;               // [V]
  double* gm;                 // [kGmresScratch] (GMRES)
  double2* kry;               // [(m + 1) * V] Krylov basis (GMRES)
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// GMRES scratch in shared memory (doubles): Hessenberg matrix, rotations, the
// rotated right-hand side g, the solution y, a flag and three reduction areas
// (16 warps at most: CTAs of <= 512 threads).
constexpr int kGmresMaxM = 20;  // longest Krylov cycle (restart length)
constexpr int kGmresMinM = 4;   // shortest one worth running
constexpr int kGmWarps = 16;
constexpr int kGmH = 0;  // [m][m+1] complex, column j at 2 j (kGmresMaxM + 1)
constexpr int kGmCs = kGmH + 2 * (kGmresMaxM + 1) * kGmresMaxM;
constexpr int kGmSn = kGmCs + kGmresMaxM;
constexpr int kGmG = kGmSn + 2 * kGmresMaxM;
constexpr int kGmY = kGmG + 2 * (kGmresMaxM + 1);
constexpr int kGmFlag = kGmY + 2 * kGmresMaxM;
constexpr int kGmR1 = kGmFlag + 2;
constexpr int kGmR2 = kGmR1 + 2 * kGmresMaxM * kGmWarps;
constexpr int kGmR3 = kGmR2 + 2 * kGmresMaxM * kGmWarps;
constexpr int kGmresScratch = kGmR3 + kGmWarps;
static_assert(kGmresScratch % 2 == 0, "the Krylov basis after the scratch must stay 16-byte aligned");

// kry_elems: complex values of the GMRES Krylov basis, 0 when the method is not GMRES
__host__ __device__ inline size_t res_smem_bytes(int ncoef, int njcoef, int N, int V, size_t kry_elems = 0) {
  size_t b = align16(sizeof(Hdr));
  b += align16(sizeof(double) * 2 * ncoef);
  b += align16(sizeof(double) * 2 * njcoef);
  b += align16(sizeof(uint32_t) * N);
  b += 2 * align16(sizeof(uint16_t) * (size_t)N * (N + 1) / 2);
  b += align16(sizeof(unsigned long long) * 48);
  b += align16(sizeof(double) * 4 * LB_MAXQ * 16);
  b += sizeof(double2) * 3 * (size_t)V;
  if (kry_elems) b += sizeof(double) * kGmresScratch + sizeof(double2) * kry_elems;
  return b;
}

__device__ ResSmem carve(unsigned char* base, int ncoef, int njcoef, int N, int V) {
  ResSmem S;
  size_t o = 0;
  S.hdr = reinterpret_cast<Hdr*>(base + o);
  o += align16(sizeof(Hdr));
  S.cu = reinterpret_cast<double*>(base + o);
  S.cd = S.cu + ncoef;
  o += align16(sizeof(double) * 2 * ncoef);
  S.jf = reinterpret_cast<double*>(base + o);
  S.ja = S.jf + njcoef;
  o += align16(sizeof(double) * 2 * njcoef);
  S.dig = reinterpret_cast<uint32_t*>(base + o);
  o += align16(sizeof(uint32_t) * N);
  S.hmap = reinterpret_cast<uint16_t*>(base + o);
  o += align16(sizeof(uint16_t) * (size_t)N * (N + 1) / 2);
  S.hmir = reinterpret_cast<uint16_t*>(base + o);
  o += align16(sizeof(uint16_t) * (size_t)N * (N + 1) / 2);
  S.slots = reinterpret_cast<unsigned long long*>(base + o);
  o += align16(sizeof(unsigned long long) * 48);
  S.red = reinterpret_cast<double*>(base + o);
  o += align16(sizeof(double) * 4 * LB_MAXQ * 16);
  S.dsm = reinterpret_cast<double2*>(base + o);
  S.zb0 = S.dsm + V;
  S.zb1 = S.zb0 + V;
  // GMRES only (present when the launch sized shared memory for it)
  S.gm = reinterpret_cast<double*>(S.zb1 + V);
  S.kry = reinterpret_cast<double2*>(S.gm + kGmresScratch);
  return S;
}

// Load constants and tables of problem P into shared memory (all threads).
// herm_ok = false keeps every element (vectors of lb_propagate may be anything).
__device__ void res_setup(const ResSmem& S, const ProbDev& P, bool herm_ok = true) {
  if (threadIdx.x == 0) {
    load_hdr(*S.hdr, P);
    if (!herm_ok) S.hdr->herm = 0;
  }
  if (herm_ok && P.herm)
    for (int i = threadIdx.x; i < P.N * (P.N + 1) / 2; i += blockDim.x) {
      const int v = P.hmap[i], k = v % P.N, l = v / P.N;
      S.hmap[i] = (uint16_t)v;
      S.hmir[i] = k != l ? (uint16_t)(l + P.N * k) : (uint16_t)0xffffu;
    }
  for (int i = threadIdx.x; i < P.ncoef; i += blockDim.x) {
    S.cu[i] = P.cu[i];
    S.cd[i] = P.cd[i];
  }
  for (int i = threadIdx.x; i < P.njcoef; i += blockDim.x) {
    S.jf[i] = P.jf[i];
    S.ja[i] = P.ja[i];
  }
  for (int i = threadIdx.x; i < P.N; i += blockDim.x) S.dig[i] = P.digits[i];
  const bool neumann = P.method == LB_SOLVER_NEUMANN;
  const double hh = 0.5 * P.h;
  for (int i = threadIdx.x; i < P.V; i += blockDim.x) {
    const double2 d = neumann ? P.D[i] : P.Dinv[i];
    S.dsm[i] = neumann ? make_double2(hh * d.x, hh * d.y) : d;
  }
  __syncthreads();
}

// vec index of this thread's element e: slot threadIdx.x + e blockDim.x of
// the CTA's element list, which with the Hermitian symmetry is the table of
// the k <= l elements (slots past it map to V, i.e. no element)
__device__ __forceinline__ int rel(const ResSmem& S, const Hdr& H, int e) {
  const int u = threadIdx.x + e * blockDim.x;
  if (!H.herm) return u;
  return u < H.Vh ? (int)S.hmap[u] : H.V;
}
// the mirror element l + N k of an off-diagonal element k + N l under the
// Hermitian symmetry (-1 otherwise)
__device__ __forceinline__ int rmirror(const Hdr& H, int v) {
  const int k = v % H.N, l = v / H.N;
  return (H.herm && k != l) ? l + H.N * k : -1;
}

// this thread's share of the merit sum for state values q[e] against t (an
// off-diagonal element under the Hermitian symmetry counts for its mirror too)
template <int E>
__device__ double merit_partial(const ResSmem& S, const Hdr& H, const double2 (&q)[E],
                                const double2* __restrict__ tar) {
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = rel(S, H, e);
    if (v < H.V) {
      const double2 t = tar[v];
      const double wm = rmirror(H, v) >= 0 ? 2.0 : 1.0;
      double x;
      if (H.kind == LB_J_FROB) {
        const double dr = q[e].x - t.x, di = q[e].y - t.y;
        x = fma(dr, dr, di * di);
      } else {
        x = fma(t.x, q[e].x, t.y * q[e].y);
      }
      acc = fma(wm, x, acc);
    }
  }
  return acc;
}

// This thread's elements, fixed for a launch: packed digits of k and l and,
// for up to two elements per thread, the vec index (V for an empty slot)
// and mirror element under the Hermitian symmetry (-1 for none) kept in
// registers; with more elements per thread those two come from the
// shared-memory tables (registers are the scarcer resource there).
template <int E>
struct Elems {
  static constexpr bool kRegs = E <= 2;
  int v[kRegs ? E : 1], m[kRegs ? E : 1];
  uint32_t kd[E], ld[E];
};

template <int E>
__device__ __forceinline__ int el_v(const Elems<E>& el, const ResSmem& S, const Hdr& H, int e) {
  if constexpr (Elems<E>::kRegs) return el.v[e];
  else return rel(S, H, e);
}
template <int E>
__device__ __forceinline__ int el_m(const Elems<E>& el, const ResSmem& S, const Hdr& H, int e) {
  if constexpr (Elems<E>::kRegs) {
    return el.m[e];
  } else {
    const int u = threadIdx.x + e * blockDim.x;
    if (!H.herm || u >= H.Vh) return -1;
    const int mm = S.hmir[u];
    return mm == 0xffff ? -1 : mm;
  }
}

template <int E>
__device__ __forceinline__ void init_elems(Elems<E>& el, const ResSmem& S, const Hdr& H) {
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = rel(S, H, e);
    if constexpr (Elems<E>::kRegs) {
      el.v[e] = v;
      el.m[e] = v < H.V ? rmirror(H, v) : -1;
    }
    if (v < H.V) {
      el.kd[e] = S.dig[v % H.N];
      el.ld[e] = S.dig[v / H.N];
    } else {
      el.kd[e] = el.ld[e] = 0;
    }
  }
}

// store x at element v of a state array and its conjugate at the mirror m (m >= 0)
__device__ __forceinline__ void rputm(double2* a, int v, int m, double2 x) {
  a[v] = x;
  if (m >= 0) a[m] = make_double2(x.x, -x.y);
}

// Per-thread plan for one element per thread and a compile-time subsystem
// count QT: the neighbour offsets and real coefficients of the element are
// time independent, so they are computed once and kept in registers; the
// inner iteration is then nothing but shared-memory loads and FP64.
template <int QT>
struct Plan {
  int o[QT][4];     // x[k+s,l], x[k,l-s], x[k-s,l], x[k,l+s]
  int ojf[QT];      // x[k+s,l+s] (decay sandwich of M)
  int oja[QT];      // x[k-s,l-s] (decay sandwich of M^+)
  double c[QT][4];  // sqrt(nk+1), sqrt(nl), sqrt(nk), sqrt(nl+1), zero off the range
  double cjf[QT], cja[QT];
  double2 d;        // this element's (I - dt/2 D)^-1 (or dt/2 D for Neumann)
};
template <>
struct Plan<0> {
  double2 d;
};

template <int QT>
__device__ void build_plan(Plan<QT>& pl, const ResSmem& S, const Hdr& H, uint32_t kd, uint32_t ld, int v) {
  const bool ok = v < H.V;
  pl.d = ok ? S.dsm[v] : make_double2(0.0, 0.0);
  if constexpr (QT > 0) {
#pragma unroll
    for (int q = 0; q < QT; ++q) {
      const int n = H.lev[q], s = H.stride[q], co = H.coff[q], sN = s * H.N;
      const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
      const int jo = H.joff[q] + nk * n + nl;
      pl.c[q][0] = ok ? S.cu[co + nk] : 0.0;
      pl.c[q][1] = ok ? S.cd[co + nl] : 0.0;
      pl.c[q][2] = ok ? S.cd[co + nk] : 0.0;
      pl.c[q][3] = ok ? S.cu[co + nl] : 0.0;
      pl.o[q][0] = ok ? v + (nk + 1 < n ? s : 0) : 0;
      pl.o[q][1] = ok ? v - (nl > 0 ? sN : 0) : 0;
      pl.o[q][2] = ok ? v - (nk > 0 ? s : 0) : 0;
      pl.o[q][3] = ok ? v + (nl + 1 < n ? sN : 0) : 0;
      pl.cjf[q] = ok && H.jump[q] != 0.0 ? S.jf[jo] : 0.0;
      pl.cja[q] = ok && H.jump[q] != 0.0 ? S.ja[jo] : 0.0;
      pl.ojf[q] = ok ? v + ((nk + 1 < n && nl + 1 < n) ? s + sN : 0) : 0;
      pl.oja[q] = ok ? v - ((nk > 0 && nl > 0) ? s + sN : 0) : 0;
    }
  }
}

// offdiag_acc with the element's plan; cq[q] = (dt/2) d_q with the sign of
// M^+ already applied for ADJ; bit q of jon set when subsystem q decays.
template <int QT, bool ADJ>
__device__ __forceinline__ void offdiag_plan(double& ar, double& ai, const double2* __restrict__ x,
                                             const Plan<QT>& pl, const double2 (&cq)[QT > 0 ? QT : 1],
                                             unsigned jon) {
#pragma unroll
  for (int q = 0; q < QT; ++q) {
    const double2 x1 = x[pl.o[q][0]];
    const double2 x2 = x[pl.o[q][1]];
    const double2 x3 = x[pl.o[q][2]];
    const double2 x4 = x[pl.o[q][3]];
    const double pr = fma(-pl.c[q][1], x2.x, pl.c[q][0] * x1.x);
    const double pi = fma(-pl.c[q][1], x2.y, pl.c[q][0] * x1.y);
    const double rr = fma(-pl.c[q][3], x4.x, pl.c[q][2] * x3.x);
    const double ri = fma(-pl.c[q][3], x4.y, pl.c[q][2] * x3.y);
    const double ur = pr + rr, ui = pi + ri, wr = pr - rr, wi = pi - ri;
    ar = fma(cq[q].y, wr, fma(cq[q].x, ui, ar));
    ai = fma(cq[q].y, wi, fma(-cq[q].x, ur, ai));
    if (jon & (1u << q)) {
      const double cj = ADJ ? pl.cja[q] : pl.cjf[q];
      const double2 x5 = x[ADJ ? pl.oja[q] : pl.ojf[q]];
      ar = fma(cj, x5.x, ar);
      ai = fma(cj, x5.y, ai);
    }
  }
}

// |x| bits, high word: enough to order magnitudes for the stopping test
__device__ __forceinline__ unsigned hi_abs(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
}
constexpr unsigned kInfHi = 0x7ff00000u;

template <int E, bool ADJ>
__device__ int res_gmres(const ResSmem& S, const Hdr& H, const Elems<E>& el, const double2* __restrict__ ct,
                         double tol);

// Solve (I - dt/2 M) z = rhs (ADJ: (I - dt/2 M^+) z = rhs) for the CTA's
// state.  Returns the iteration count (>= 1), -1 when max_iter is reached,
// -2 on NaN/Inf.  On return, zbuf[cur] holds z; every thread has passed the
// final barrier.  The stopping test compares the high words of the bit
// patterns, hi(max|z_new - z|) < hi(rtol max|rhs|), which implies the exact
// test and is taken identically by every thread (and in a recompute).
// QT > 0 (with E == 1) uses the per-thread plan.  GM: the kernel variant
// that can also run GMRES (res_gmres) when the problem's method asks for it;
// the fixed-point kernels are compiled without it.
template <int E, int QT, bool ADJ, bool GM = false>
__device__ int res_solve(const ResSmem& S, const Hdr& H, const Elems<E>& el, const Plan<QT>& pl,
                         const double2 (&rhs)[E], const double2* __restrict__ ct, double fac, int& cur,
                         const double2* pc = nullptr) {
  static_assert(QT == 0 || E == 1, "the per-thread plan holds one element");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool neumann = H.method == LB_SOLVER_NEUMANN;
  const bool gmres = GM && H.method == LB_SOLVER_GMRES;
  const int V = H.V, maxit = H.max_iter;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  unsigned* slots = reinterpret_cast<unsigned*>(S.slots);
  double2 cq[QT > 0 ? QT : 1];
  unsigned jon = 0;
  if constexpr (QT > 0) {
#pragma unroll
    for (int q = 0; q < QT; ++q) {
      const double2 c = ct[q];
      cq[q] = ADJ ? make_double2(-c.x, -c.y) : c;
      jon |= H.jump[q] != 0.0 ? (1u << q) : 0u;
    }
  }
  unsigned qmax = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = el_v(el, S, H, e);
    if (v < V) {
      double2 z0 = rhs[e];
      if (!neumann) {
        const double2 d = QT > 0 ? pl.d : S.dsm[v];
        const double di = ADJ ? -d.y : d.y;
        const double ur = pc ? rhs[e].x + pc[e].x : rhs[e].x, ui = pc ? rhs[e].y + pc[e].y : rhs[e].y;
        z0 = make_double2(fma(d.x, ur, -di * ui), fma(d.x, ui, di * ur));
      }
      rputm(S.zb0, v, el_m(el, S, H, e), z0);
      if (gmres) S.zb1[v] = rhs[e];
      qmax = max(qmax, max(hi_abs(rhs[e].x), hi_abs(rhs[e].y)));
    }
  }
  qmax = __reduce_max_sync(kFull, qmax);
  if (lane == 0) slots[64 + warp] = qmax;
  __syncthreads();
  qmax = 0;
  for (int w = 0; w < nwarps; ++w) qmax = max(qmax, slots[64 + w]);
  if (qmax >= kInfHi) return -2;
  // rtol * (a value <= max|rhs|), so the test is never looser than the exact one
  const double tol = H.rtol * __longlong_as_double(static_cast<long long>((unsigned long long)qmax << 32));
  cur = 0;
  if constexpr (GM) {
    if (gmres) return res_gmres<E, ADJ>(S, H, el, ct, tol);
  }
  const unsigned thr = hi_abs(tol * fac);
  for (int it = 0; it < maxit; ++it) {
    const double2* __restrict__ zc = cur ? S.zb1 : S.zb0;
    double2* __restrict__ zn = cur ? S.zb0 : S.zb1;
    unsigned dmax = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      if (v < V) {
        double ar = rhs[e].x, ai = rhs[e].y;
        double2 d;
        if constexpr (QT > 0) {
          offdiag_plan<QT, ADJ>(ar, ai, zc, pl, cq, jon);
          d = pl.d;
        } else {
          offdiag_acc<ADJ>(ar, ai, zc, v, el.kd[e], el.ld[e], H, T, ct);
          d = S.dsm[v];
        }
        const double di = ADJ ? -d.y : d.y;
        const double2 zo = zc[v];
        double2 z;
        if (!neumann) {
          z.x = fma(d.x, ar, -di * ai);
          z.y = fma(d.x, ai, di * ar);
        } else {
          z.x = ar + fma(d.x, zo.x, -di * zo.y);
          z.y = ai + fma(d.x, zo.y, di * zo.x);
        }
        rputm(zn, v, el_m(el, S, H, e), z);
        dmax = max(dmax, max(hi_abs(z.x - zo.x), hi_abs(z.y - zo.y)));
      }
    }
    dmax = __reduce_max_sync(kFull, dmax);
    if (lane == 0) slots[(it & 1) * 32 + warp] = dmax;
    __syncthreads();
    dmax = 0;
    for (int w = 0; w < nwarps; ++w) dmax = max(dmax, slots[(it & 1) * 32 + w]);
    cur ^= 1;
    if (dmax >= kInfHi) return -2;
    if (dmax < thr) return it + 1;
  }
  return -1;
}

// Predictor of the first iterate for one CTA's state: the corrections of the
// previous steps live in the ring P.hist ([kPredOrder][M * V], this state's
// elements at base + v); every element is read and written by the thread that
// owns it, so no synchronisation is needed.
template <int E>
struct Pred {
  double2* hist = nullptr;
  const double2* D = nullptr;
  size_t stride = 0;
  double hh = 0.0;
  int n = 0, slot = 0;
  __device__ void init(const ProbDev& P, size_t base) {
    hist = P.hist + base;
    D = P.D;
    stride = (size_t)P.M * P.V;
    hh = 0.5 * P.h;
    n = slot = 0;
  }
  __device__ void predict(double2 (&pc)[E], const Elems<E>& el, const ResSmem& S, const Hdr& H, int V) const {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      double pr = 0.0, pi = 0.0;
      if (v < V) {
        int sl = slot;
        if (n == kPredOrder) {
          // steady state: all terms, loads issued together
#pragma unroll
          for (int i = 1; i <= kPredOrder; ++i) {
            sl = sl > 0 ? sl - 1 : kPredOrder - 1;
            const double2 c = hist[(size_t)sl * stride + v];
            pr = fma(kExtrap[kPredOrder][i - 1], c.x, pr);
            pi = fma(kExtrap[kPredOrder][i - 1], c.y, pi);
          }
        } else {
          for (int i = 1; i <= n; ++i) {
            sl = sl > 0 ? sl - 1 : kPredOrder - 1;
            const double w = kExtrap[n][i - 1];
            const double2 c = hist[(size_t)sl * stride + v];
            pr = fma(w, c.x, pr);
            pi = fma(w, c.y, pi);
          }
        }
      }
      pc[e] = make_double2(pr, pi);
    }
  }
  template <bool ADJ>
  __device__ void record(const double2* zc, const double2 (&rhs)[E], const Elems<E>& el, const ResSmem& S,
                         const Hdr& H, int V) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      if (v < V) {
        const double2 z = zc[v], d = __ldg(D + v);
        const double dr = hh * d.x, di = hh * (ADJ ? -d.y : d.y);
        hist[(size_t)slot * stride + v] = make_double2(z.x - fma(dr, z.x, -di * z.y) - rhs[e].x,
                                                       z.y - fma(dr, z.y, di * z.x) - rhs[e].y);
      }
    }
    n = n < kPredOrder ? n + 1 : kPredOrder;
    slot = slot + 1 < kPredOrder ? slot + 1 : 0;
  }
};

// Deterministic CTA sum of one double per thread; the result is returned to
// every thread.  Uses S.red[0..15] and two barriers.
__device__ double cta_sum(const ResSmem& S, double x) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  x = warp_sum(x);
  if (lane == 0) S.red[warp] = x;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nwarps; ++w) t += S.red[w];
  __syncthreads();
  return t;
}

// ---------------------------------------------------------------------------
// GMRES inner solve (the paper's Krylov method, Sec. IV), one CTA per state.
//
// Restarted GMRES(m) on the Jacobi-preconditioned system
//   K z = b,   K = I - Dinv (dt/2) O,   b = Dinv q
// (ADJ: conj(Dinv) and the adjoint off-diagonal part), equivalent to
// (I - dt/2 M) z = q.  Its residual b - K z = Dinv (q + dt/2 O z) - z is the
// increment of one Jacobi sweep, the quantity the fixed-point test bounds.
// Arnoldi uses classical Gram-Schmidt with one re-orthogonalisation pass; all
// dot products and norms are fixed-order CTA reductions, so a recompute
// reproduces every iterate bit for bit.  Thread 0 applies the Givens
// rotations and solves the small triangular system.  A cycle stops when the
// rotated residual norm |g_{j+1}| = ||b - K z||_2 (which bounds the largest
// component) falls below tol; a restart recomputes the residual from z.
// Iterations counted: products with O (Arnoldi steps plus one per restart).
// On entry zb0 holds the first iterate z_0 and zb1 the right-hand side q; on a
// converged return zb0 holds z and every thread has passed a barrier.
template <int E, bool ADJ>
__device__ int res_gmres(const ResSmem& S, const Hdr& H, const Elems<E>& el, const double2* __restrict__ ct,
                         double tol) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int V = H.V, m = H.krylov;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  double* gm = S.gm;
  double2* kry = S.kry;
  const double2* rhs = S.zb1;
  double2* xs = S.zb0;
  double2 x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = threadIdx.x + e * blockDim.x;
    x[e] = v < V ? xs[v] : make_double2(0.0, 0.0);
  }
  int its = 0;
  for (;;) {
    // r = Dinv (q + dt/2 O z) - z, normalised into the first basis vector
    double nrm = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = threadIdx.x + e * blockDim.x;
      if (v < V) {
        double ar = rhs[v].x, ai = rhs[v].y;
        offdiag_acc<ADJ>(ar, ai, xs, v, el.kd[e], el.ld[e], H, T, ct);
        const double2 d = S.dsm[v];
        const double di = ADJ ? -d.y : d.y;
        const double2 r = make_double2(fma(d.x, ar, -di * ai) - x[e].x, fma(d.x, ai, di * ar) - x[e].y);
        kry[v] = r;
        nrm = fma(r.x, r.x, fma(r.y, r.y, nrm));
      }
    }
    ++its;
    const double beta = sqrt(cta_sum(S, nrm));
    if (!(beta <= 1.0e300)) return -2;  // NaN or Inf
    if (beta < tol) return its;         // z (in zb0) already passed a barrier
    if (its >= H.max_iter) return -1;
    const double ib = 1.0 / beta;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = threadIdx.x + e * blockDim.x;
      if (v < V) kry[v] = make_double2(kry[v].x * ib, kry[v].y * ib);
    }
    if (threadIdx.x == 0) {
      gm[kGmG] = beta;
      gm[kGmG + 1] = 0.0;
    }
    int k = 0;
    bool conv = false;
    for (int j = 0; j < m; ++j) {
      __syncthreads();  // v_j complete
      const double2* vj = kry + (size_t)j * V;
      double2* vn = kry + (size_t)(j + 1) * V;
      // w = K v_j
      double2 w[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = threadIdx.x + e * blockDim.x;
        w[e] = make_double2(0.0, 0.0);
        if (v < V) {
          double ar = 0.0, ai = 0.0;
          offdiag_acc<ADJ>(ar, ai, vj, v, el.kd[e], el.ld[e], H, T, ct);
          const double2 d = S.dsm[v];
          const double di = ADJ ? -d.y : d.y;
          const double2 u = vj[v];
          w[e] = make_double2(u.x - fma(d.x, ar, -di * ai), u.y - fma(d.x, ai, di * ar));
        }
      }
      // h = V_j^H w, w -= V_j h; twice
      double* hc = gm + kGmH + 2 * j * (kGmresMaxM + 1);
      for (int pass = 0; pass < 2; ++pass) {
        double* red = gm + (pass ? kGmR2 : kGmR1);
        for (int i = 0; i <= j; ++i) {
          double sr = 0.0, si = 0.0;
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int v = threadIdx.x + e * blockDim.x;
            if (v < V) {
              const double2 u = kry[(size_t)i * V + v];
              sr = fma(u.x, w[e].x, fma(u.y, w[e].y, sr));
              si = fma(u.x, w[e].y, fma(-u.y, w[e].x, si));
            }
          }
          const double t = warp_sum2(sr, si, lane);
          if ((lane & 15) == 0) red[(2 * i + (lane >> 4)) * kGmWarps + warp] = t;
        }
        __syncthreads();
        for (int i = 0; i <= j; ++i) {
          double hr = 0.0, hi = 0.0;
          for (int ww = 0; ww < nw; ++ww) {
            hr += red[(2 * i) * kGmWarps + ww];
            hi += red[(2 * i + 1) * kGmWarps + ww];
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int v = threadIdx.x + e * blockDim.x;
            if (v < V) {
              const double2 u = kry[(size_t)i * V + v];
              w[e].x -= fma(hr, u.x, -hi * u.y);
              w[e].y -= fma(hr, u.y, hi * u.x);
            }
          }
          if (threadIdx.x == 0) {
            hc[2 * i] = pass ? hc[2 * i] + hr : hr;
            hc[2 * i + 1] = pass ? hc[2 * i + 1] + hi : hi;
          }
        }
      }
      double n2 = 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) n2 = fma(w[e].x, w[e].x, fma(w[e].y, w[e].y, n2));
      n2 = warp_sum(n2);
      if (lane == 0) gm[kGmR3 + warp] = n2;
      __syncthreads();
      double s2 = 0.0;
      for (int ww = 0; ww < nw; ++ww) s2 += gm[kGmR3 + ww];
      const double hn = sqrt(s2);
      if (!(hn <= 1.0e300)) return -2;
      const double ih = hn > 0.0 ? 1.0 / hn : 0.0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = threadIdx.x + e * blockDim.x;
        if (v < V) vn[v] = make_double2(w[e].x * ih, w[e].y * ih);
      }
      ++its;
      k = j + 1;
      if (threadIdx.x == 0) {
        // earlier rotations on column j, then the one that zeroes h_{j+1,j}
        for (int i = 0; i < j; ++i) {
          const double c = gm[kGmCs + i], sr = gm[kGmSn + 2 * i], si = gm[kGmSn + 2 * i + 1];
          const double ar = hc[2 * i], ai = hc[2 * i + 1], br = hc[2 * i + 2], bi = hc[2 * i + 3];
          // (a, b) <- (c a + s b, -conj(s) a + c b)
          hc[2 * i] = c * ar + (sr * br - si * bi);
          hc[2 * i + 1] = c * ai + (sr * bi + si * br);
          hc[2 * i + 2] = c * br - (sr * ar + si * ai);
          hc[2 * i + 3] = c * bi - (sr * ai - si * ar);
        }
        const double ar = hc[2 * j], ai = hc[2 * j + 1];
        const double na = hypot(ar, ai), r = hypot(na, hn);
        double c, sr, si;
        if (r == 0.0) {
          c = 1.0, sr = 0.0, si = 0.0;
        } else if (na == 0.0) {
          c = 0.0, sr = 1.0, si = 0.0;
          hc[2 * j] = hn;
          hc[2 * j + 1] = 0.0;
        } else {
          // c = |a|/r, s = (a/|a|) h/r, rho = (a/|a|) r
          c = na / r;
          sr = ar / na * (hn / r);
          si = ai / na * (hn / r);
          hc[2 * j] = ar / na * r;
          hc[2 * j + 1] = ai / na * r;
        }
        hc[2 * j + 2] = 0.0;
        hc[2 * j + 3] = 0.0;
        gm[kGmCs + j] = c;
        gm[kGmSn + 2 * j] = sr;
        gm[kGmSn + 2 * j + 1] = si;
        const double gr = gm[kGmG + 2 * j], gi = gm[kGmG + 2 * j + 1];
        // (g_j, g_{j+1}) <- (c g_j, -conj(s) g_j)
        gm[kGmG + 2 * j] = c * gr;
        gm[kGmG + 2 * j + 1] = c * gi;
        const double nr = -(sr * gr + si * gi), ni = -(sr * gi - si * gr);
        gm[kGmG + 2 * j + 2] = nr;
        gm[kGmG + 2 * j + 3] = ni;
        gm[kGmFlag] = (hypot(nr, ni) < tol || hn == 0.0) ? 1.0 : 0.0;
      }
      __syncthreads();
      conv = gm[kGmFlag] != 0.0;
      if (conv || its >= H.max_iter) break;
    }
    // z += V_k y with R y = g (back substitution by thread 0)
    if (threadIdx.x == 0) {
      bool bad = false;
      for (int i = k - 1; i >= 0; --i) {
        double tr = gm[kGmG + 2 * i], ti = gm[kGmG + 2 * i + 1];
        for (int l = i + 1; l < k; ++l) {
          const double* hl = gm + kGmH + 2 * l * (kGmresMaxM + 1);
          const double yr = gm[kGmY + 2 * l], yi = gm[kGmY + 2 * l + 1];
          tr -= hl[2 * i] * yr - hl[2 * i + 1] * yi;
          ti -= hl[2 * i] * yi + hl[2 * i + 1] * yr;
        }
        const double* hi_ = gm + kGmH + 2 * i * (kGmresMaxM + 1);
        const double dr = hi_[2 * i], dim = hi_[2 * i + 1];
        const double den = dr * dr + dim * dim;
        gm[kGmY + 2 * i] = (tr * dr + ti * dim) / den;
        gm[kGmY + 2 * i + 1] = (ti * dr - tr * dim) / den;
        bad = bad || !(fabs(gm[kGmY + 2 * i]) <= 1.0e300 && fabs(gm[kGmY + 2 * i + 1]) <= 1.0e300);
      }
      gm[kGmFlag + 1] = bad ? 1.0 : 0.0;
    }
    __syncthreads();
    if (gm[kGmFlag + 1] != 0.0) return -2;  // singular triangle or overflow
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = threadIdx.x + e * blockDim.x;
      if (v < V) {
        double2 z = x[e];
        for (int i = 0; i < k; ++i) {
          const double yr = gm[kGmY + 2 * i], yi = gm[kGmY + 2 * i + 1];
          const double2 u = kry[(size_t)i * V + v];
          z.x += fma(yr, u.x, -yi * u.y);
          z.y += fma(yr, u.y, yi * u.x);
        }
        x[e] = z;
        xs[v] = z;
      }
    }
    __syncthreads();
    if (conv) return its;
    if (its >= H.max_iter) return -1;
  }
}

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

// ---------------------------------------------------------------------------
// forward sweep, one CTA per (problem, state) work item

template <int E, int QT, bool GM>
__global__ void __launch_bounds__(512) k_forward_res(const ProbDev* __restrict__ probs,
                                                     const WorkItem* __restrict__ items, int tape) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WorkItem wi = items[blockIdx.x];
  const ProbDev& P = probs[wi.prob];
  const int i = wi.state;
  const ResSmem S = carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  res_setup(S, P);
  const Hdr& H = *S.hdr;
  const int V = H.V;  // kept in a register: H is reloaded after every barrier
  Elems<E> el;
  init_elems<E>(el, S, H);
  Plan<QT> pl;
  build_plan<QT>(pl, S, H, el.kd[0], el.ld[0], rel(S, H, 0));
  const size_t base = (size_t)i * H.V;
  double2 q[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = el_v(el, S, H, e);
    q[e] = v < V ? P.q0[base + v] : make_double2(0.0, 0.0);
  }
  CtaStats stats;
  // predictor only when no step is ever recomputed (K == 0): recomputed stage
  // vectors then stay bit-identical to the forward ones
  const bool pred = H.K == 0 && H.method != LB_SOLVER_NEUMANN;
  Pred<E> pr;
  if (pred) pr.init(P, base);
  double2 pc[E];
  // running penalty sum_j dt beta(t_j) J(q^j) (Sec. III, eq. optimproblem)
  double jpen = 0.0;
  for (int j = 0; j < H.NT; ++j) {
    if (H.gamma1 != 0.0) jpen = fma(P.pen[j], merit_value(H.kind, cta_sum(S, merit_partial<E>(S, H, q, P.tar + base))), jpen);
    if (tape && H.K > 0 && j % H.K == 0) {
      double2* ck = P.ckpt + ((size_t)i * H.n_ckpt + j / H.K) * H.V;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = el_v(el, S, H, e);
        if (v < V) ck[v] = q[e];
      }
    }
    int cur;
    if (pred) pr.predict(pc, el, S, H, V);
    const int it = res_solve<E, QT, false, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur,
                                                 pred ? pc : nullptr);
    if (it < 0) {
      if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
      stats.flush(P.status);
      return;
    }
    stats.add(0, it);
    const double2* zc = cur ? S.zb1 : S.zb0;
    if (pred) pr.template record<false>(zc, q, el, S, H, V);
    double2* tp = (tape && H.K == 0) ? P.ckpt + ((size_t)i * H.NT + j) * H.V : nullptr;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      if (v < V) {
        const double2 z = zc[v];
        if (tp) tp[v] = z;
        // q^{j+1} = q^j + dt M z = 2 z - q^j  (eq. IMR with eq. linsystem_primal)
        q[e] = make_double2(fma(2.0, z.x, -q[e].x), fma(2.0, z.y, -q[e].y));
      }
    }
  }
  // final state and merit functional (Sec. III)
  double acc = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = el_v(el, S, H, e);
    if (v < V) {
      rputm(P.qT + base, v, el_m(el, S, H, e), q[e]);
      const double2 t = P.tar[base + v];
      // an off-diagonal element under the symmetry stands for its mirror too
      const double wm = el_m(el, S, H, e) >= 0 ? 2.0 : 1.0;
      if (H.kind == LB_J_FROB) {
        const double dr = q[e].x - t.x, di = q[e].y - t.y;
        if (wm == 1.0)
          acc = fma(dr, dr, fma(di, di, acc));
        else
          acc = fma(wm, fma(dr, dr, di * di), acc);
      } else {
        if (wm == 1.0)
          acc = fma(t.x, q[e].x, fma(t.y, q[e].y, acc));
        else
          acc = fma(wm, fma(t.x, q[e].x, t.y * q[e].y), acc);
      }
    }
  }
  const double tot = cta_sum(S, acc);
  if (threadIdx.x == 0) P.J[i] = merit_value(H.kind, tot) + H.gamma1 * jpen;
  stats.flush(P.status);
}

// ---------------------------------------------------------------------------
// backward sweep: recompute each checkpoint segment, then adjoint steps with
// the gradient pieces of eq. reducedgradient.

template <int E, int QT, bool GM>
__global__ void __launch_bounds__(512) k_backward_res(const ProbDev* __restrict__ probs,
                                                      const WorkItem* __restrict__ items) {
  extern __shared__ __align__(16) unsigned char smem[];
  const WorkItem wi = items[blockIdx.x];
  const ProbDev& P = probs[wi.prob];
  const int i = wi.state;
  const ResSmem S = carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  res_setup(S, P);
  const Hdr& H = *S.hdr;
  const int V = H.V;  // kept in a register: H is reloaded after every barrier
  Elems<E> el;
  init_elems<E>(el, S, H);
  Plan<QT> pl;
  build_plan<QT>(pl, S, H, el.kd[0], el.ld[0], rel(S, H, 0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const size_t base = (size_t)i * H.V;
  const double w = P.wgt[i];
  const double wt = linear_sign(P.kind) * w;
  // terminal condition qhat^{N_T} = beta_i/M g_i (Appendix B): g = q - q_tar
  // for J_Frob, g = -q_tar for J_Tr
  double2 lam[E], qf[E];
  // running penalty: q^j is rebuilt backwards, q^j = 2 z^j - q^{j+1}, in the
  // workspace buffer qb (each thread its own elements), starting from q^{N_T}
  if (H.gamma1 != 0.0)
    for (int v = threadIdx.x; v < V; v += blockDim.x) P.qb[base + v] = P.qT[base + v];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = el_v(el, S, H, e);
    lam[e] = make_double2(0.0, 0.0);
    qf[e] = lam[e];
    if (v < V) {
      const double2 t = P.tar[base + v];
      if (H.kind == LB_J_FROB) {
        const double2 qq = P.qT[base + v];
        lam[e] = make_double2(w * (qq.x - t.x), w * (qq.y - t.y));
      } else {
        lam[e] = make_double2(wt * t.x, wt * t.y);
      }
    }
  }
  CtaStats stats;
  const int nseg = H.K > 0 ? (H.NT + H.K - 1) / H.K : 1;
  // adjoint predictor: the adjoint steps come in the same order for every K
  const bool apred = H.method != LB_SOLVER_NEUMANN;
  Pred<E> pr;
  if (apred) pr.init(P, base);
  double2 pc[E];
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int j0 = H.K > 0 ? sg * H.K : 0;
    const int j1 = H.K > 0 ? min(H.NT, j0 + H.K) : H.NT;
    if (H.K > 0) {
      // recompute the stage vectors z^j of this segment from its checkpoint
      const double2* ck = P.ckpt + ((size_t)i * H.n_ckpt + sg) * H.V;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = el_v(el, S, H, e);
        if (v < V) qf[e] = ck[v];
      }
      for (int j = j0; j < j1; ++j) {
        int cur;
        const int it = res_solve<E, QT, false, GM>(S, H, el, pl, qf, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur);
        if (it < 0) {
          if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
          stats.flush(P.status);
          return;
        }
        stats.add(1, it);
        const double2* zc = cur ? S.zb1 : S.zb0;
        double2* sgv = P.seg + ((size_t)i * H.K + (j - j0)) * H.V;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int v = el_v(el, S, H, e);
          if (v < V) {
            const double2 z = zc[v];
            sgv[v] = z;
            qf[e] = make_double2(fma(2.0, z.x, -qf[e].x), fma(2.0, z.y, -qf[e].y));
          }
        }
      }
    }
    for (int j = j1 - 1; j >= j0; --j) {
      const double2* ct = P.ctab + (size_t)j * H.cq;
      int cur;
      // (I - dt/2 (M^{j+1/2})^+) zhat^j = qhat^{j+1}   (eq. linsystem_adjoint)
      if (apred) pr.predict(pc, el, S, H, V);
      const int it = res_solve<E, QT, true, GM>(S, H, el, pl, lam, ct, stop_factor(P, j), cur, apred ? pc : nullptr);
      if (it < 0) {
        if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
        stats.flush(P.status);
        return;
      }
      stats.add(2, it);
      const double2* zh = cur ? S.zb1 : S.zb0;
      if (apred) pr.template record<true>(zh, lam, el, S, H, V);
      const double2* Zt = H.K > 0 ? P.seg + ((size_t)i * H.K + (j - j0)) * H.V : P.ckpt + ((size_t)i * H.NT + j) * H.V;
      // gradient pieces (eq. reducedgradient): for every subsystem q,
      //   g_a  = zhat^H vec(-i[a_q, Z])   = -i sum_kl Z_kl conj(R_zhat)
      //   g_ad = zhat^H vec(-i[a_q^+, Z]) = -i sum_kl Z_kl conj(P_zhat)
      // (index shift of the commutator onto zhat), with P, R as in offdiag_acc.
      double2 Z[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = el_v(el, S, H, e);
        Z[e] = v < V ? Zt[v] : make_double2(0.0, 0.0);
      }
      for (int q = 0; q < H.Q; ++q) {
        const int n = H.lev[q], s = H.stride[q], co = H.coff[q], sN = s * H.N;
        double sar = 0.0, sai = 0.0, sdr = 0.0, sdi = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int v = el_v(el, S, H, e);
          if (v < V) {
            const int nk = (el.kd[e] >> (H.db * q)) & H.dm, nl = (el.ld[e] >> (H.db * q)) & H.dm;
            const double c1 = S.cu[co + nk], c2 = S.cd[co + nl], c3 = S.cd[co + nk], c4 = S.cu[co + nl];
            const double2 x1 = zh[v + (nk + 1 < n ? s : 0)];
            const double2 x2 = zh[v - (nl > 0 ? sN : 0)];
            const double2 x3 = zh[v - (nk > 0 ? s : 0)];
            const double2 x4 = zh[v + (nl + 1 < n ? sN : 0)];
            const double pr = fma(-c2, x2.x, c1 * x1.x);
            const double pi = fma(-c2, x2.y, c1 * x1.y);
            const double rr = fma(-c4, x4.x, c3 * x3.x);
            const double ri = fma(-c4, x4.y, c3 * x3.y);
            // Z conj(R) and Z conj(P)
            if (el_m(el, S, H, e) < 0) {
              sar = fma(Z[e].x, rr, fma(Z[e].y, ri, sar));
              sai = fma(Z[e].y, rr, fma(-Z[e].x, ri, sai));
              sdr = fma(Z[e].x, pr, fma(Z[e].y, pi, sdr));
              sdi = fma(Z[e].y, pr, fma(-Z[e].x, pi, sdi));
            } else {
              // Hermitian Z and zhat: the mirror element (l, k) adds -conj(B) to
              // the g_a sum and -conj(A) to the g_ad sum, A = Z conj(R), B = Z conj(P)
              const double ar = fma(Z[e].x, rr, Z[e].y * ri), ai = fma(Z[e].y, rr, -Z[e].x * ri);
              const double br = fma(Z[e].x, pr, Z[e].y * pi), bi = fma(Z[e].y, pr, -Z[e].x * pi);
              sar += ar - br;
              sai += ai + bi;
              sdr += br - ar;
              sdi += bi + ai;
            }
          }
        }
        const double r = warp_sum4(sar, sai, sdr, sdi, lane);
        if ((lane & 7) == 0) S.red[(q * 4 + (lane >> 3)) * 16 + warp] = r;
      }
      __syncthreads();
      if (threadIdx.x < 4 * H.Q) {
        double t = 0.0;
        for (int ww = 0; ww < nwarps; ++ww) t += S.red[threadIdx.x * 16 + ww];
        const int q = threadIdx.x >> 2, c = threadIdx.x & 3;
        // multiply by -i: g = (S.im, -S.re)
        double* g = reinterpret_cast<double*>(P.gproj + (((size_t)i * H.NT + j) * H.Q + q) * 2);
        if (c == 0) g[1] = -t;
        if (c == 1) g[0] = t;
        if (c == 2) g[3] = -t;
        if (c == 3) g[2] = t;
      }
      // qhat^j = qhat^{j+1} + dt M^+ zhat = 2 zhat - qhat^{j+1}, plus the running
      // penalty's source gamma1 beta_i/M dt beta(t_j) g(q^j) (Appendix B)
      const double pw = H.gamma1 != 0.0 ? H.gamma1 * w * P.pen[j] : 0.0;
      const double ls = linear_sign(H.kind);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int v = el_v(el, S, H, e);
        if (v < V) {
          const double2 z = zh[v];
          lam[e] = make_double2(fma(2.0, z.x, -lam[e].x), fma(2.0, z.y, -lam[e].y));
          if (H.gamma1 != 0.0) {
            const double2 qn = P.qb[base + v], t = P.tar[base + v];
            const double2 qj = make_double2(fma(2.0, Z[e].x, -qn.x), fma(2.0, Z[e].y, -qn.y));
            P.qb[base + v] = qj;
            if (H.kind == LB_J_FROB) {
              lam[e].x = fma(pw, qj.x - t.x, lam[e].x);
              lam[e].y = fma(pw, qj.y - t.y, lam[e].y);
            } else {
              lam[e].x = fma(pw * ls, t.x, lam[e].x);
              lam[e].y = fma(pw * ls, t.y, lam[e].y);
            }
          }
        }
      }
    }
  }
  stats.flush(P.status);
}

// ---------------------------------------------------------------------------
// propagate given vectors (tests and the step-level API), one CTA per vector

template <int E, int QT, bool GM>
__global__ void __launch_bounds__(512) k_propagate_res(const ProbDev* __restrict__ pp, int adjoint, int j0, int j1,
                                                       double2* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ProbDev& P = *pp;
  const ResSmem S = carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  res_setup(S, P, false);
  const Hdr& H = *S.hdr;
  const int V = H.V;  // kept in a register: H is reloaded after every barrier
  Elems<E> el;
  init_elems<E>(el, S, H);
  Plan<QT> pl;
  build_plan<QT>(pl, S, H, el.kd[0], el.ld[0], rel(S, H, 0));
  double2* xv = x + (size_t)blockIdx.x * H.V;
  double2 q[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = threadIdx.x + e * blockDim.x;
    q[e] = v < V ? xv[v] : make_double2(0.0, 0.0);
  }
  CtaStats stats;
  for (int jj = 0; jj < j1 - j0; ++jj) {
    const int j = adjoint ? j1 - 1 - jj : j0 + jj;
    int cur;
    const int it = adjoint ? res_solve<E, QT, true, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur)
                           : res_solve<E, QT, false, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur);
    if (it < 0) {
      if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
      stats.flush(P.status);
      return;
    }
    stats.add(adjoint ? 2 : 0, it);
    const double2* zc = cur ? S.zb1 : S.zb0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = threadIdx.x + e * blockDim.x;
      if (v < V) {
        const double2 z = zc[v];
        q[e] = make_double2(fma(2.0, z.x, -q[e].x), fma(2.0, z.y, -q[e].y));
      }
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = threadIdx.x + e * blockDim.x;
    if (v < V) xv[v] = q[e];
  }
  stats.flush(P.status);
}


// ---------------------------------------------------------------------------
// cluster-split sweeps for small states (latency-bound time loops)
//
// One state per thread-block cluster of C CTAs.  Each element's off-diagonal
// work is split over L = 2Q lanes: lane r handles half r%2 of subsystem r/2
// of the commutator (P = sqrt(nk+1) x[k+s,l] - sqrt(nl) x[k,l-s] or
// R = sqrt(nk) x[k-s,l] - sqrt(nl+1) x[k,l+s]) times its complex control
// factor, the P half also the decay sandwich; every lane runs the same
// instructions on its own data.  The L partial sums meet through shuffles,
// and a CTA holds at most 4 warps (one per SM sub-partition).
//
// Every CTA keeps a full replica of the iterate and the diagonal tables in
// shared memory; each element's right-hand side lives in the registers of
// the lanes that own it.  An inner iteration ends without any cluster-wide
// barrier: each element's new value, and each warp's largest change, are
// pushed into every CTA with st.async, whose completion is counted in bytes
// on the receiving CTA's mbarrier (one per exchange parity, so a CTA one
// exchange ahead never disturbs the current phase); each CTA waits only for
// its own mbarrier, with a bounded wait.  All CTAs see the same data and
// take the same decisions.  The next step's first iterate travels with the
// inner iterations' pushes (cl_iterate), so a step that converges in one
// inner iteration needs one exchange.

// Lanes per element: 2QT (one half P or R of a subsystem each, and the two
// halves U and W of each Jaynes-Cummings pair: QT = Q + pairs), or with CS
// ("component split") 4QT, two lanes per half, one for the real and one for
// the imaginary part of its contribution; rounded up to a power of two.
template <int QT, bool CS = false>
struct ClLanes {
  static constexpr int L = CS ? (4 * QT <= 4 ? 4 : (4 * QT <= 8 ? 8 : 16)) : (2 * QT <= 2 ? 2 : (2 * QT <= 4 ? 4 : 8));
};

constexpr long long kMbarSpinLimit = 1LL << 24;



__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned mapa_u32(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_async_f64x2(unsigned addr, double x, double y, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "d"(x), "d"(y), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void st_async_u32(unsigned addr, unsigned v, unsigned mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr), "r"(v),
               "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned mbar, unsigned tx) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

struct ClSmem {
  Hdr* hdr;
  double* cu;
  double* cd;
  double* jf;
  double* ja;
  uint32_t* dig;
  double2* zb;               // [2][V] replicated iterate, indexed by exchange parity
  double2* zs;               // [2][V] next step's first iterate, pushed with each inner iteration, by step parity
  double2* dv;               // [V] (I - dt/2 D)^-1, or dt/2 D for Neumann
  double2* dm;               // [V] I - dt/2 D
  double2* ch;               // [kPredOrder][V] ring of the previous steps' off-diagonal corrections
  unsigned* dsl;             // [2][64] per exchange parity: warp maxima of |z_new - z| (index cta * 4 + warp),
                             // then of the next step's |rhs| (32 + cta * 4 + warp)
  unsigned long long* mbar;  // [2]
  double* gred;              // [8 units][4 warps][2]
};

__host__ __device__ inline size_t cl_smem_bytes(int ncoef, int njcoef, int N, int V) {
  size_t b = align16(sizeof(Hdr));
  b += align16(sizeof(double) * 2 * ncoef);
  b += align16(sizeof(double) * 2 * njcoef);
  b += align16(sizeof(uint32_t) * N);
  b += sizeof(double2) * (6 + kPredOrder) * (size_t)V;
  b += align16(sizeof(unsigned) * 128);
  b += align16(sizeof(unsigned long long) * 2);
  b += align16(sizeof(double) * 64);
  return b;
}

__device__ ClSmem cl_carve(unsigned char* base, int ncoef, int njcoef, int N, int V) {
  ClSmem S;
  size_t o = 0;
  S.hdr = reinterpret_cast<Hdr*>(base + o);
  o += align16(sizeof(Hdr));
  S.cu = reinterpret_cast<double*>(base + o);
  S.cd = S.cu + ncoef;
  o += align16(sizeof(double) * 2 * ncoef);
  S.jf = reinterpret_cast<double*>(base + o);
  S.ja = S.jf + njcoef;
  o += align16(sizeof(double) * 2 * njcoef);
  S.dig = reinterpret_cast<uint32_t*>(base + o);
  o += align16(sizeof(uint32_t) * N);
  S.zb = reinterpret_cast<double2*>(base + o);
  S.zs = S.zb + 2 * (size_t)V;
  S.dv = S.zs + 2 * (size_t)V;
  S.dm = S.dv + V;
  S.ch = S.dm + V;
  o += sizeof(double2) * (6 + kPredOrder) * (size_t)V;
  S.dsl = reinterpret_cast<unsigned*>(base + o);
  o += align16(sizeof(unsigned) * 128);
  S.mbar = reinterpret_cast<unsigned long long*>(base + o);
  o += align16(sizeof(unsigned long long) * 2);
  S.gred = reinterpret_cast<double*>(base + o);
  return S;
}

// Per-CTA set-up; ends with a cluster barrier, so no CTA pushes into another
// before its shared memory and mbarriers are initialised.
__device__ void cl_setup(const ClSmem& S, const ProbDev& P, cg::cluster_group& cl) {
  if (threadIdx.x == 0) load_hdr(*S.hdr, P);
  for (int i = threadIdx.x; i < P.ncoef; i += blockDim.x) {
    S.cu[i] = P.cu[i];
    S.cd[i] = P.cd[i];
  }
  for (int i = threadIdx.x; i < P.njcoef; i += blockDim.x) {
    S.jf[i] = P.jf[i];
    S.ja[i] = P.ja[i];
  }
  for (int i = threadIdx.x; i < P.N; i += blockDim.x) S.dig[i] = P.digits[i];
  const bool neumann = P.method == LB_SOLVER_NEUMANN;
  const double hh = 0.5 * P.h;
  for (int i = threadIdx.x; i < P.V; i += blockDim.x) {
    const double2 D = P.D[i];
    S.dv[i] = neumann ? make_double2(hh * D.x, hh * D.y) : P.Dinv[i];
    S.dm[i] = make_double2(1.0 - hh * D.x, -(hh * D.y));
  }
  for (int i = threadIdx.x; i < 128; i += blockDim.x) S.dsl[i] = 0u;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&S.mbar[0]), 1);
    mbar_init(smem_u32(&S.mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  cl.sync();
}

// one lane's share of one element
struct ClPlan {
  int v;        // element (vec index) of this lane; 0 when none
  bool ev;      // the lane belongs to a real element
  int r;        // lane within the element, 0..L-1
  int q;        // subsystem of this lane's half (0 for padding lanes)
  bool rhalf;   // R half (else P half)
  bool act;     // the lane has a half (not a padding lane)
  int oa, ob, ojf, oja;
  double ca, cb, cjf, cja;
  double2 d;    // the element's entry of S.dv
  double2 dmv;  // the element's entry of S.dm
  // problem constants the inner loops use, kept in registers (shared memory
  // values are reloaded after every asm statement that clobbers memory)
  int V, maxit;
  bool neu;     // Neumann iteration
  double rtol;
};

template <int QT, bool CS>
__device__ ClPlan cl_plan(const ClSmem& S, int C, int crank) {
  constexpr int L = ClLanes<QT, CS>::L;
  const Hdr& H = *S.hdr;
  const int Vc = (H.V + C - 1) / C;
  const int le = threadIdx.x / L;
  ClPlan pl;
  pl.r = threadIdx.x % L;
  const int v = crank * Vc + le;
  pl.ev = le < Vc && v < H.V;
  pl.v = pl.ev ? v : 0;
  const int hv = CS ? (pl.r >> 1) : pl.r;  // half index of this lane
  const int u = hv < 2 * QT ? hv : -1;
  pl.act = pl.ev && u >= 0;
  pl.q = u >= 0 ? u / 2 : 0;
  pl.rhalf = u >= 0 && (u & 1);
  pl.oa = pl.ob = pl.ojf = pl.oja = pl.v;
  pl.ca = pl.cb = pl.cjf = pl.cja = 0.0;
  pl.d = pl.ev ? S.dv[v] : make_double2(0.0, 0.0);
  pl.dmv = pl.ev ? S.dm[v] : make_double2(0.0, 0.0);
  pl.V = H.V;
  pl.maxit = H.max_iter;
  pl.neu = H.method == LB_SOLVER_NEUMANN;
  pl.rtol = H.rtol;
  if (pl.ev && u >= 0 && pl.q >= H.Q) {
    // Jaynes-Cummings pair k (Sec. II) as two more halves: U with the factor
    // (dt/2) G (like a P half) and W with its conjugate (like an R half),
    //   U = sqrt(np_k) sqrt(nq_k+1) x[k-sp+sq, l] - sqrt(np_l+1) sqrt(nq_l) x[k, l+sp-sq]
    //   W = sqrt(np_k+1) sqrt(nq_k) x[k+sp-sq, l] - sqrt(np_l) sqrt(nq_l+1) x[k, l-sp+sq]
    // (a coefficient is zero where its neighbour leaves the range)
    const uint32_t kd = S.dig[v % H.N], ld = S.dig[v / H.N];
    const int k = pl.q - H.Q, p = H.jp[k], q = H.jq[k];
    const int np = H.lev[p], nq = H.lev[q], d = H.stride[q] - H.stride[p], cp = H.coff[p], cqo = H.coff[q];
    const int pk = (kd >> (H.db * p)) & H.dm, qk = (kd >> (H.db * q)) & H.dm;
    const int plv = (ld >> (H.db * p)) & H.dm, ql = (ld >> (H.db * q)) & H.dm;
    if (!pl.rhalf) {
      pl.ca = S.cd[cp + pk] * S.cu[cqo + qk];
      pl.oa = v + ((pk > 0 && qk + 1 < nq) ? d : 0);
      pl.cb = S.cu[cp + plv] * S.cd[cqo + ql];
      pl.ob = v - ((ql > 0 && plv + 1 < np) ? d * H.N : 0);
    } else {
      pl.ca = S.cu[cp + pk] * S.cd[cqo + qk];
      pl.oa = v - ((qk > 0 && pk + 1 < np) ? d : 0);
      pl.cb = S.cd[cp + plv] * S.cu[cqo + ql];
      pl.ob = v + ((plv > 0 && ql + 1 < nq) ? d * H.N : 0);
    }
  } else if (pl.ev && u >= 0) {
    const uint32_t kd = S.dig[v % H.N], ld = S.dig[v / H.N];
    const int q = pl.q, n = H.lev[q], s = H.stride[q], co = H.coff[q], sN = s * H.N;
    const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
    if (!pl.rhalf) {
      pl.oa = v + (nk + 1 < n ? s : 0);
      pl.ob = v - (nl > 0 ? sN : 0);
      pl.ca = S.cu[co + nk];
      pl.cb = S.cd[co + nl];
      if (H.jump[q] != 0.0) {
        const int jo = H.joff[q] + nk * n + nl;
        pl.cjf = S.jf[jo];
        pl.cja = S.ja[jo];
        pl.ojf = v + ((nk + 1 < n && nl + 1 < n) ? s + sN : 0);
        pl.oja = v - ((nk > 0 && nl > 0) ? s + sN : 0);
      }
    } else {
      pl.oa = v - (nk > 0 ? s : 0);
      pl.ob = v + (nl + 1 < n ? sN : 0);
      pl.ca = S.cd[co + nk];
      pl.cb = S.cu[co + nl];
    }
  }
  return pl;
}

// iteration and mbarrier phase counters; identical in every thread of the cluster
struct ClCount {
  unsigned gk = 0;                // inner iterations so far (selects buffer and mbarrier parity)
  unsigned ph = 0u;               // bit b: completed phases of mbar[b] (mod 2)
};

// Predictor of the off-diagonal correction c = (I - dt/2 D) z - rhs of a step:
// the polynomial extrapolation through the last n recorded corrections,
// c_j ~ sum_i (-1)^(i+1) binom(n, i) c_{j-i}, n = min(steps recorded,
// kPredOrder).  hist.slot is where the next correction will be recorded.
struct ClHist {
  bool on = false;  // the sweep uses the predictor
  int n = 0;        // corrections recorded so far (capped at kPredOrder)
  int slot = 0;     // ring position of the next record
  __device__ void advance() {
    n = n < kPredOrder ? n + 1 : kPredOrder;
    slot = slot + 1 < kPredOrder ? slot + 1 : 0;
  }
};
__device__ __forceinline__ ClHist cl_hist_on() {
  ClHist h;
  h.on = true;
  return h;
}

// Cluster addresses an inner iteration uses, fixed for a launch: per buffer
// parity, this lane's element in CTA pl.r (its first store target) with that
// CTA's mbarrier, and this warp's maximum slot in CTA `lane` with that CTA's
// mbarrier.
struct ClAddr {
  unsigned zb[2], zs[2], mb[2], dsl[2], qsl[2], mbl[2];
};
__device__ ClAddr cl_addr(const ClSmem& S, const ClPlan& pl, int C, int crank) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int V = S.hdr->V;
  const unsigned rr0 = pl.r < C ? pl.r : 0, lr = lane < C ? lane : 0;
  ClAddr A;
  for (int b = 0; b < 2; ++b) {
    A.zb[b] = mapa_u32(smem_u32(S.zb + (size_t)b * V + pl.v), rr0);
    A.mb[b] = mapa_u32(smem_u32(&S.mbar[b]), rr0);
    A.zs[b] = mapa_u32(smem_u32(S.zs + (size_t)b * V + pl.v), rr0);
    A.dsl[b] = mapa_u32(smem_u32(S.dsl + 64 * b + crank * 4 + warp), lr);
    A.qsl[b] = mapa_u32(smem_u32(S.dsl + 64 * b + 32 + crank * 4 + warp), lr);
    A.mbl[b] = mapa_u32(smem_u32(&S.mbar[b]), lr);
  }
  return A;
}

// the control factors, stop factor and running-penalty weight of one step,
// loaded a step ahead
struct ClStep {
  double2 c;   // d_q or its Jaynes-Cummings factor for this lane's half
  double fac;  // stopping-test factor
  double pen;  // dt beta(t_j) of the running penalty (0 without one)
};
// where they come from, resolved once per launch and kept in registers (the
// problem record is in global memory and is reloaded after every asm
// statement that clobbers memory)
struct ClSrc {
  const double2* ct;  // control table, this lane's column
  const double* sf;   // stop factors, or null (factor 1)
  const double* pen;  // running-penalty weights, or null (no penalty)
  int cq;             // control table entries per step
};
__device__ __forceinline__ ClSrc cl_src(const ProbDev& P, const ClPlan& pl, int cq) {
  ClSrc src;
  src.ct = P.ctab + pl.q;
  src.sf = P.method == LB_SOLVER_JACOBI ? P.sfac : nullptr;
  src.pen = P.gamma1 != 0.0 ? P.pen : nullptr;
  src.cq = cq;
  return src;
}
__device__ __forceinline__ ClStep cl_step(const ClSrc& src, int j) {
  ClStep st;
  st.c = src.ct[(size_t)j * src.cq];
  st.fac = src.sf ? src.sf[j] : 1.0;
  st.pen = src.pen ? src.pen[j] : 0.0;
  return st;
}

// One exchange.  Lanes with pl.ev && pl.r < C push this lane's element
// value z into every CTA's next buffer (the element's lanes share the C
// stores), and one lane per CTA pushes this warp's maximum of m into that
// CTA's slot.  With `spec` the lanes also push zn, the element's first
// iterate for the next step, into spec buffer sb, and the warp's maximum of
// mn into the second slot set.  Then wait (bounded) for every CTA's pushes.
// Returns 0 with the largest slot values in mmax (and mnmax), or -3 if a wait
// gave up; the vote keeps a timeout, should one ever happen, a decision of
// the whole CTA.
template <int L>
__device__ __forceinline__ int cl_exchange(const ClSmem& S, const ClPlan& pl, const ClAddr& A, double2 z,
                                           unsigned m, int C, ClCount& cnt, unsigned& mmax, bool spec = false,
                                           int sb = 0, double2 zn = double2(), unsigned mn = 0u,
                                           unsigned* mnmax = nullptr) {
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int V = pl.V;
  const unsigned p = (cnt.gk + 1) & 1;
  const unsigned mb_local = smem_u32(&S.mbar[p]);
  const unsigned per = (unsigned)V * 16u + (unsigned)(C * nwarps) * 4u;
  if (threadIdx.x == 0) mbar_arrive_expect_tx(mb_local, spec ? 2u * per : per);
  if (pl.ev && pl.r < C) {
    st_async_f64x2(A.zb[p], z.x, z.y, A.mb[p]);
    if (spec) st_async_f64x2(A.zs[sb], zn.x, zn.y, A.mb[p]);
    const unsigned dst = smem_u32(S.zb + (size_t)p * V + pl.v);
    const unsigned dsp = smem_u32(S.zs + (size_t)sb * V + pl.v);
    for (int cc = pl.r + L; cc < C; cc += L) {
      const unsigned mbr = mapa_u32(mb_local, cc);
      st_async_f64x2(mapa_u32(dst, cc), z.x, z.y, mbr);
      if (spec) st_async_f64x2(mapa_u32(dsp, cc), zn.x, zn.y, mbr);
    }
  }
  m = __reduce_max_sync(kFull, m);
  if (spec) mn = __reduce_max_sync(kFull, mn);
  if (lane < C) {
    st_async_u32(A.dsl[p], m, A.mbl[p]);
    if (spec) st_async_u32(A.qsl[p], mn, A.mbl[p]);
  }
  long long spins = 0;
  int timed_out = 0;
  while (!mbar_try_wait(mb_local, (cnt.ph >> p) & 1u)) {
    if (++spins > kMbarSpinLimit) {
      timed_out = 1;
      break;
    }
  }
  if (__syncthreads_or(timed_out)) return -3;
  cnt.ph ^= 1u << p;
  ++cnt.gk;
  // slot cta * 4 + warp of each set: one per lane, reduced across the warp
  const unsigned* d = S.dsl + p * 64;
  const bool has = lane < 4 * C;
  mmax = __reduce_max_sync(kFull, has ? d[lane] : 0u);
  if (spec) *mnmax = __reduce_max_sync(kFull, has ? d[32 + lane] : 0u);
  return 0;
}

// Every lane of an element holds the element's complex values; lane r
// computes component r & 1 (imaginary when odd) of each new one.
__device__ __forceinline__ double cl_comp(const ClPlan& pl, double2 x) { return (pl.r & 1) ? x.y : x.x; }
__device__ __forceinline__ double2 cl_join(const ClPlan& pl, double c) {
  const double o = __shfl_xor_sync(kFull, c, 1);
  return (pl.r & 1) ? make_double2(o, c) : make_double2(c, o);
}

// rc + the predicted correction, this lane's component: the terms of the
// extrapolation (hist h, the step being predicted) are split among the
// element's lanes of that component and summed over them; term 0 is `c0`
// when has_c0 (the correction just recorded), else read from the ring.
template <int L>
__device__ __forceinline__ double cl_predicted(const ClSmem& S, const ClPlan& pl, double rc, ClHist h, bool has_c0,
                                               double c0) {
  constexpr int LH = L / 2;
  const int hh = pl.r >> 1, odd = pl.r & 1, n = h.n, V = pl.V;
  const double* ring = reinterpret_cast<const double*>(S.ch);
  double acc = hh == 0 ? rc : 0.0;
#pragma unroll
  for (int k = 0; k < (kPredOrder + LH - 1) / LH; ++k) {
    const int t = hh + k * LH;
    if (t < n) {
      int sl = h.slot - 1 - t;
      if (sl < 0) sl += kPredOrder;
      const double c = (t == 0 && has_c0) ? c0 : ring[2 * ((size_t)sl * V + pl.v) + odd];
      acc = fma(kExtrap[n][t], c, acc);
    }
  }
#pragma unroll
  for (int o = 2; o < L; o <<= 1) acc += __shfl_xor_sync(kFull, acc, o);
  return acc;
}

// Start of a step: the first iterate of this lane's element from its
// right-hand side (this lane's component rc): rc itself (Neumann), else
// (I - dt/2 D)^-1 (rhs + predicted correction), no correction before the
// first recorded step; pushed to every CTA with max |rhs|, which comes back
// in qmax.  Returns 0 or -3 (a wait gave up).
template <int L, bool ADJ>
__device__ __forceinline__ double cl_first_comp(const ClSmem& S, const ClPlan& pl, double rc, ClHist h, bool has_c0,
                                                double c0) {
  if (pl.neu) return rc;
  const double u = h.n > 0 ? cl_predicted<L>(S, pl, rc, h, has_c0, c0) : rc;
  const double di = ADJ ? -pl.d.y : pl.d.y;
  // real: d.x ur - di ui, imaginary: d.x ui + di ur
  return fma(pl.d.x, u, ((pl.r & 1) ? di : -di) * __shfl_xor_sync(kFull, u, 1));
}

template <int QT, bool ADJ, bool CS>
__device__ int cl_start(const ClSmem& S, const ClPlan& pl, const ClAddr& A, double rc, ClHist h, bool has_c0,
                        double c0, int C, ClCount& cnt, unsigned& qmax) {
  constexpr int L = ClLanes<QT, CS>::L;
  const double2 z0 = cl_join(pl, cl_first_comp<L, ADJ>(S, pl, rc, h, has_c0, c0));
  const unsigned m = (pl.ev && pl.r < 2) ? hi_abs(rc) : 0u;
  return cl_exchange<L>(S, pl, A, z0, m, C, cnt, qmax);
}

// End of a step for this lane's element, given its z: this lane's
// component of c_j = (I - dt/2 D) z - rhs (predictor on; returned in cc) and
// of the next right-hand side 2 z - rhs + src (returned; src is the lane's
// component of the adjoint's running-penalty source, else 0).  cl_commit
// records cc in ring slot h.slot once the step has converged.
template <bool ADJ, bool SRC = false>
__device__ __forceinline__ double cl_update(const ClPlan& pl, double2 z, double2 rhs, ClHist h, double& cc,
                                            double src = 0.0) {
  const int odd = pl.r & 1;
  const double zc = odd ? z.y : z.x, zo = odd ? z.x : z.y, rc = odd ? rhs.y : rhs.x;
  if (h.on) {
    const double b = ADJ ? -pl.dmv.y : pl.dmv.y;
    // real: dm.x z.x - b z.y - r.x, imaginary: dm.x z.y + b z.x - r.y
    cc = fma(pl.dmv.x, zc, fma(odd ? b : -b, zo, -rc));
  }
  // SRC: a source term exists (its addition is compiled out otherwise)
  if constexpr (SRC) return fma(2.0, zc, -rc) + src;
  return fma(2.0, zc, -rc);
}
__device__ __forceinline__ void cl_commit(const ClSmem& S, const ClPlan& pl, ClHist h, double cc) {
  if (h.on && pl.ev && pl.r < 2)
    reinterpret_cast<double*>(S.ch)[2 * ((size_t)h.slot * pl.V + pl.v) + (pl.r & 1)] = cc;
}

// What a converged inner solve hands to the next step when it pushed the
// next step's first iterate speculatively: this lane's components of c_j
// and of the next right-hand side, and max |next rhs| over the cluster.
struct ClNext {
  double cc = 0.0, rn = 0.0;
  unsigned qmax = 0u;
};

// Inner iterations of (I - dt/2 M) z = rhs (ADJ: M^+) for the cluster's
// state from the first iterate in buffer (gk & 1); `rhs` is this lane's
// element of the right-hand side and qmax the high word of max |rhs|.
// Returns the iteration count, -1 (max_iter), -2 (NaN/Inf) or -3 (a wait
// gave up).  On success S.zb + (gk & 1) * V holds z in every CTA, and zout
// the lane's element of it.
//
// The first iteration reads the first iterate from z0 (the buffer cl_start
// or the previous step's speculative push filled).  With `spec` (a next step
// follows) every iteration also pushes the first iterate of the next step
// computed from its own z as if it were the converged one (hist hn: the
// predictor state of the next step), into spec buffer sb, so a step that
// converges needs no further exchange; nx returns what the next step needs.
template <int QT, bool ADJ, bool CS, bool SRC = false>
__device__ int cl_iterate(const ClSmem& S, const ClPlan& pl, const ClAddr& A, const double2* z0, double2 rhs,
                          ClStep st, unsigned qmax, int C, ClCount& cnt, double2& zout, bool spec = false,
                          ClHist hn = ClHist(), int sb = 0, ClNext* nx = nullptr, double src = 0.0) {
  constexpr int L = ClLanes<QT, CS>::L;
  const int V = pl.V;
  const bool neumann = pl.neu;
  if (qmax >= kInfHi) return -2;
  const unsigned thr =
      hi_abs(pl.rtol * __longlong_as_double(static_cast<long long>((unsigned long long)qmax << 32)) * st.fac);
  // this lane's complex factor: -i d P -> (b - i a) P, -i conj(d) R -> (-b - i a) R
  const double2 c = st.c;
  double Ar = pl.rhalf ? -c.y : c.y, Ai = -c.x;
  if (ADJ) {
    Ar = -Ar;
    Ai = -Ai;
  }
  const double di = ADJ ? -pl.d.y : pl.d.y;
  const bool odd = pl.r & 1;  // this lane's component (imaginary)
  const double sdi = odd ? di : -di;
  const double2 r0 = pl.r == 0 ? rhs : make_double2(0.0, 0.0);
  // CS: this lane's component of U xa + W xb, U = A ca, W = -A cb (real:
  // U.r xa.x - U.i xa.y + W.r xb.x - W.i xb.y; imaginary: U.r xa.y + U.i xa.x
  // + W.r xb.y + W.i xb.x), started from rhs on the two lanes of half 0
  const double u1 = Ar * pl.ca, u2 = odd ? Ai * pl.ca : -(Ai * pl.ca);
  const double u3 = -(Ar * pl.cb), u4 = odd ? -(Ai * pl.cb) : Ai * pl.cb;
  const double init = pl.r < 2 ? (odd ? rhs.y : rhs.x) : 0.0;
  const double cj = ADJ ? pl.cja : pl.cjf;
  const int oj = ADJ ? pl.oja : pl.ojf;
  for (int it = 0; it < pl.maxit; ++it) {
    const double2* __restrict__ zc = it == 0 ? z0 : S.zb + (size_t)(cnt.gk & 1) * V;
    const double2 xa = zc[pl.oa], xb = zc[pl.ob], x5 = zc[oj], zo = zc[pl.v];
    double k;
    if constexpr (CS) {
      k = fma(u1, odd ? xa.y : xa.x,
              fma(u2, odd ? xa.x : xa.y, fma(u3, odd ? xb.y : xb.x, fma(u4, odd ? xb.x : xb.y,
                                                                       fma(cj, odd ? x5.y : x5.x, init)))));
      // sum over the halves: lanes of the same component
#pragma unroll
      for (int o = 2; o < L; o <<= 1) k += __shfl_xor_sync(kFull, k, o);
    } else {
      const double xr = fma(-pl.cb, xb.x, pl.ca * xa.x);
      const double xi = fma(-pl.cb, xb.y, pl.ca * xa.y);
      // lane 0 of the element starts from the right-hand side
      double accr = fma(Ar, xr, fma(-Ai, xi, r0.x));
      double acci = fma(Ar, xi, fma(Ai, xr, r0.y));
      accr = fma(cj, x5.x, accr);
      acci = fma(cj, x5.y, acci);
      // Sum over the element's L lanes with one component per lane: after the
      // first exchange even lanes carry the real and odd lanes the imaginary
      // part, so each level costs one FP64 add.
      k = odd ? acci : accr;
      k += __shfl_xor_sync(kFull, odd ? accr : acci, 1);
#pragma unroll
      for (int o = 2; o < L; o <<= 1) k += __shfl_xor_sync(kFull, k, o);
    }
    const double am = k;  // this lane's component of rhs + dt/2 O z
    const double zom = odd ? zo.y : zo.x;
    double zm;
    if (!neumann) {
      // real: d.x ar - di ai, imaginary: d.x ai + di ar
      zm = fma(pl.d.x, am, sdi * __shfl_xor_sync(kFull, am, 1));
    } else {
      zm = am + fma(pl.d.x, zom, sdi * __shfl_xor_sync(kFull, zom, 1));
    }
    const double2 z = cl_join(pl, zm);
    const unsigned dm = (pl.ev && pl.r < 2) ? hi_abs(zm - zom) : 0u;
    unsigned dmax;
    if (spec) {
      double cc = 0.0;
      const double rn = cl_update<ADJ, SRC>(pl, z, rhs, hn, cc, src);
      const double2 zn = cl_join(pl, cl_first_comp<L, ADJ>(S, pl, rn, hn, true, cc));
      const unsigned qn = (pl.ev && pl.r < 2) ? hi_abs(rn) : 0u;
      unsigned qnmax = 0u;
      if (cl_exchange<L>(S, pl, A, z, dm, C, cnt, dmax, true, sb, zn, qn, &qnmax)) return -3;
      nx->cc = cc;
      nx->rn = rn;
      nx->qmax = qnmax;
    } else if (cl_exchange<L>(S, pl, A, z, dm, C, cnt, dmax)) {
      return -3;
    }
    if (dmax >= kInfHi) return -2;
    if (dmax < thr) {
      zout = z;
      return it + 1;
    }
  }
  return -1;
}

__device__ __forceinline__ int cl_code(int it) { return it == -1 ? LB_ENOTCONV : (it == -2 ? LB_ENAN : LB_ECUDA); }

// A step's work in every sweep below: the first iterate is in every CTA
// (pushed by cl_start at a sweep's or segment's start, else by the previous
// step's inner iterations along with their iterates), the step's constants
// were loaded one step ahead, and cl_iterate converges; a step that
// converges in one inner iteration costs one exchange.  Each element's
// right-hand side lives in the registers of its own lanes; only iterates
// travel between the CTAs.

// J_i over the cluster: this CTA's own elements (lanes r == 0), summed per
// CTA in a fixed order and gathered in CTA 0's shared memory; the cluster
// barrier that follows makes them visible there.
//
// With the running penalty each own lane also holds pacc, the sum over the
// steps of dt beta(t_j) f(q^j) for its element (f the merit summand), which
// is summed the same way into the second slot set.
template <bool PEN>
__device__ void cl_objective_part(const ClSmem& S, const ClPlan& pl, const ProbDev& P, size_t base, double2 q,
                                  int crank, double pacc) {
  const Hdr& H = *S.hdr;
  double acc = 0.0;
  if (pl.ev && pl.r == 0) {
    P.qT[base + pl.v] = q;
    const double2 t = P.tar[base + pl.v];
    if (H.kind == LB_J_FROB) {
      const double dr = q.x - t.x, dq = q.y - t.y;
      acc = fma(dr, dr, dq * dq);
    } else {
      acc = fma(t.x, q.x, t.y * q.y);
    }
  }
  acc = warp_sum(acc);
  const double pw = PEN ? warp_sum(pacc) : 0.0;
  if ((threadIdx.x & 31) == 0) {
    S.gred[threadIdx.x >> 5] = acc;
    S.gred[8 + (threadIdx.x >> 5)] = pw;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, u = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t += S.gred[w];
      u += S.gred[8 + w];
    }
    const unsigned dst = mapa_u32(smem_u32(&S.gred[32 + crank]), 0);
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(dst), "d"(t) : "memory");
    const unsigned dsu = mapa_u32(smem_u32(&S.gred[48 + crank]), 0);
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(dsu), "d"(u) : "memory");
  }
}

// the merit summand f of this lane's element for state value q and target t
__device__ __forceinline__ double cl_merit_summand(int kind, double2 q, double2 t) {
  if (kind == LB_J_FROB) {
    const double dr = q.x - t.x, dq = q.y - t.y;
    return fma(dr, dr, dq * dq);
  }
  return fma(t.x, q.x, t.y * q.y);
}

// PEN: the running penalty (a separate instantiation, so that the sweeps
// without it keep their registers)
template <int QT, bool CS, bool PEN>
__global__ void __launch_bounds__(128, 1) k_forward_cl(const ProbDev* __restrict__ pp, int tape) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const ProbDev& P = *pp;
  const int C = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int i = blockIdx.x / C;
  const ClSmem S = cl_carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  cl_setup(S, P, cl);
  const Hdr& H = *S.hdr;
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank);
  const ClAddr A = cl_addr(S, pl, C, crank);
  const ClSrc src = cl_src(P, pl, H.cq);
  const size_t base = (size_t)i * H.V;
  const bool own = pl.ev && pl.r == 0;  // the lane that writes the element's tapes
  const int NT = H.NT, K = H.K, V = H.V;
  // this lane's element in the checkpoints (K > 0) or the stage tape (K == 0), step 0
  double2* const tp0 = P.ckpt + (K > 0 ? (size_t)i * H.n_ckpt * V : (size_t)i * NT * V) + pl.v;
  double2 rhs = P.q0[base + pl.v];
  // running penalty gamma1 sum_j dt beta(t_j) J(q^j) (Sec. III, eq. optimproblem):
  // J is affine in the merit sum, so each own lane accumulates
  // sum_j dt beta(t_j) f(q^j) for its element, and ppen = sum_j dt beta(t_j)
  constexpr bool penal = PEN;
  const double2 tv = penal && own ? P.tar[base + pl.v] : make_double2(0.0, 0.0);
  double pacc = 0.0, ppen = 0.0;
  ClCount cnt;
  CtaStats stats;
  bool failed = false;
  // the predictor is used only when no step is ever recomputed (K == 0), so
  // recomputed stage vectors stay bit-identical to the forward ones
  const bool pred = H.K == 0 && H.method != LB_SOLVER_NEUMANN;
  ClHist hist = pred ? cl_hist_on() : ClHist();
  unsigned qmax = 0;
  if (cl_start<QT, false, CS>(S, pl, A, cl_comp(pl, rhs), hist, false, 0.0, C, cnt, qmax)) {
    if (threadIdx.x == 0 && crank == 0) record_error(P.status, LB_ECUDA, 0);
    failed = true;
  }
  const double2* z0 = S.zb + (size_t)(cnt.gk & 1) * H.V;
  ClStep nx = cl_step(src, 0);
  for (int j = 0; j < NT && !failed; ++j) {
    if (tape && K > 0 && j % K == 0 && own) tp0[(size_t)(j / K) * V] = rhs;
    const ClStep st = nx;
    if (j + 1 < NT) nx = cl_step(src, j + 1);
    if (penal) {
      if (own) pacc = fma(st.pen, cl_merit_summand(H.kind, rhs, tv), pacc);
      ppen += st.pen;
    }
    ClHist hn = hist;
    if (hist.on) hn.advance();
    const bool spec = j + 1 < NT;
    ClNext nxt;
    double2 z;
    const int it = cl_iterate<QT, false, CS>(S, pl, A, z0, rhs, st, qmax, C, cnt, z, spec, hn, (j + 1) & 1, &nxt);
    if (it < 0) {
      if (threadIdx.x == 0 && crank == 0) record_error(P.status, cl_code(it), j);
      failed = true;
      break;
    }
    if (crank == 0) stats.add(0, it);
    if (tape && K == 0 && own) tp0[(size_t)j * V] = z;
    // q^{j+1} = 2 z - q^j; the next step's first iterate is already in every CTA
    if (spec) {
      cl_commit(S, pl, hist, nxt.cc);
      rhs = cl_join(pl, nxt.rn);
      qmax = nxt.qmax;
      z0 = S.zs + (size_t)((j + 1) & 1) * V;
    } else {
      double cc = 0.0;
      rhs = cl_join(pl, cl_update<false>(pl, z, rhs, hist, cc));
    }
    hist = hn;
  }
  if (!failed) cl_objective_part<PEN>(S, pl, P, base, rhs, crank, pacc);
  stats.flush(P.status);
  cl.sync();  // the partial sums are in CTA 0; no CTA leaves while another may still push into it
  if (!failed && crank == 0 && threadIdx.x == 0) {
    double t = 0.0, u = 0.0;
    for (int c = 0; c < C; ++c) {
      t += S.gred[32 + c];
      u += S.gred[48 + c];
    }
    double J = merit_value(H.kind, t);
    // sum_j pen_j merit(S_j) = a sum_j pen_j S_j + b sum_j pen_j for merit(S) = a S + b
    if (penal) J += H.gamma1 * (merit_value(H.kind, u) - merit_value(H.kind, 0.0) + merit_value(H.kind, 0.0) * ppen);
    P.J[i] = J;
  }
}

template <int QT, bool CS, bool PEN>
__global__ void __launch_bounds__(128, 1) k_backward_cl(const ProbDev* __restrict__ pp) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  constexpr int L = ClLanes<QT, CS>::L;
  const ProbDev& P = *pp;
  const int C = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int i = blockIdx.x / C;
  const ClSmem S = cl_carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  cl_setup(S, P, cl);
  const Hdr& H = *S.hdr;
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank);
  const ClAddr A = cl_addr(S, pl, C, crank);
  const ClSrc src = cl_src(P, pl, H.cq);
  const int V = H.V, K = H.K, NT = H.NT, Qn = H.Q;  // in registers: H is reloaded after every asm clobber
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const size_t base = (size_t)i * V;
  const double w = P.wgt[i];
  const double wt = linear_sign(P.kind) * w;
  // terminal condition qhat^{N_T} = beta_i/M g_i (Appendix B), this lane's element
  double2 ll;
  {
    const double2 t = P.tar[base + pl.v];
    if (H.kind == LB_J_FROB) {
      const double2 qq = P.qT[base + pl.v];
      ll = make_double2(w * (qq.x - t.x), w * (qq.y - t.y));
    } else {
      ll = make_double2(wt * t.x, wt * t.y);
    }
  }
  ClCount cnt;
  CtaStats stats;
  bool failed = false;
  const int nseg = K > 0 ? (NT + K - 1) / K : 1;
  // the adjoint sweep visits the steps in the same order for every K, and
  // its first iterates are the same arithmetic whether formed at a segment
  // start or at the end of the previous step, so its results never depend
  // on the checkpoint interval
  ClHist ahist = H.method != LB_SOLVER_NEUMANN ? cl_hist_on() : ClHist();
  ClHist none;
  const bool own = pl.ev && pl.r == 0;
  // running penalty: its adjoint source gamma1 beta_i/M dt beta(t_j) g(q^j)
  // (Appendix B) needs q^j, rebuilt backwards q^j = 2 z^j - q^{j+1} from the
  // stage vectors, starting from q^{N_T}, in the registers of each element's lanes
  constexpr bool penal = PEN;
  const double g1w = H.gamma1 * w, ls = linear_sign(H.kind);
  const int kind = H.kind;
  const double2 tv = penal ? P.tar[base + pl.v] : make_double2(0.0, 0.0);
  double2 qb = penal ? P.qT[base + pl.v] : make_double2(0.0, 0.0);
  // gradient pieces of this warp go to state slot (i * C + crank) * nwarps + warp of gproj
  double2* gbase = P.gproj + (size_t)((i * C + crank) * nwarps + warp) * NT * Qn * 2;
  for (int sg = nseg - 1; sg >= 0 && !failed; --sg) {
    const int j0 = K > 0 ? sg * K : 0;
    const int j1 = K > 0 ? min(NT, j0 + K) : NT;
    if (K > 0) {
      double2 rr = P.ckpt[((size_t)i * H.n_ckpt + sg) * V + pl.v];
      unsigned qr = 0;
      if (cl_start<QT, false, CS>(S, pl, A, cl_comp(pl, rr), none, false, 0.0, C, cnt, qr)) {
        if (threadIdx.x == 0 && crank == 0) record_error(P.status, LB_ECUDA, j0);
        failed = true;
        break;
      }
      const double2* z0r = S.zb + (size_t)(cnt.gk & 1) * V;
      ClStep nx = cl_step(src, j0);
      for (int j = j0; j < j1; ++j) {
        const ClStep st = nx;
        if (j + 1 < j1) nx = cl_step(src, j + 1);
        const bool spec = j + 1 < j1;
        ClNext nxt;
        double2 z;
        const int it = cl_iterate<QT, false, CS>(S, pl, A, z0r, rr, st, qr, C, cnt, z, spec, none, (j + 1) & 1, &nxt);
        if (it < 0) {
          if (threadIdx.x == 0 && crank == 0) record_error(P.status, cl_code(it), j);
          failed = true;
          break;
        }
        if (crank == 0) stats.add(1, it);
        if (own) P.seg[((size_t)i * K + (j - j0)) * V + pl.v] = z;
        if (spec) {
          rr = cl_join(pl, nxt.rn);
          qr = nxt.qmax;
          z0r = S.zs + (size_t)((j + 1) & 1) * V;
        }
      }
      if (failed) break;
      __syncthreads();  // segment tape written by each element's lane r = 0 before its other lanes read it
    }
    unsigned qmax = 0;
    if (cl_start<QT, true, CS>(S, pl, A, cl_comp(pl, ll), ahist, false, 0.0, C, cnt, qmax)) {
      if (threadIdx.x == 0 && crank == 0) record_error(P.status, LB_ECUDA, j1 - 1);
      failed = true;
      break;
    }
    const double2* z0 = S.zb + (size_t)(cnt.gk & 1) * V;
    ClStep nx = cl_step(src, j1 - 1);
    // this lane's stage vector element of step j, loaded one step ahead so
    // that its latency is hidden behind a whole step
    const bool gl = pl.act;
    const bool zl = gl || (penal && pl.ev);  // lanes that need the stage vector
    const double2* tape = K > 0 ? P.seg + (size_t)i * K * V : P.ckpt + (size_t)i * NT * V;
    const int jt = K > 0 ? j0 : 0;  // tape row of step j is j - jt
    double2 Znx = zl ? tape[(size_t)(j1 - 1 - jt) * V + pl.v] : make_double2(0.0, 0.0);
    for (int j = j1 - 1; j >= j0; --j) {
      const double2 Z = Znx;
      if (zl && j > j0) Znx = tape[(size_t)(j - 1 - jt) * V + pl.v];
      const ClStep st = nx;
      if (j > j0) nx = cl_step(src, j - 1);
      // this lane's component of the penalty source, added to qhat^j
      double psrc = 0.0;
      if (penal) {
        const double2 qj = make_double2(fma(2.0, Z.x, -qb.x), fma(2.0, Z.y, -qb.y));
        qb = qj;
        const double gc = kind == LB_J_FROB ? cl_comp(pl, qj) - cl_comp(pl, tv) : ls * cl_comp(pl, tv);
        psrc = (g1w * st.pen) * gc;
      }
      ClHist hn = ahist;
      if (ahist.on) hn.advance();
      const bool spec = j > j0;
      ClNext nxt;
      double2 zh;
      const int it =
          cl_iterate<QT, true, CS, PEN>(S, pl, A, z0, ll, st, qmax, C, cnt, zh, spec, hn, (j - 1) & 1, &nxt, psrc);
      if (it < 0) {
        if (threadIdx.x == 0 && crank == 0) record_error(P.status, cl_code(it), j);
        failed = true;
        break;
      }
      if (crank == 0) stats.add(2, it);
      const double2* zb = S.zb + (size_t)(cnt.gk & 1) * V;
      // gradient piece of this lane's half (eq. reducedgradient): sum_kl Z conj(X_zhat),
      // X the half's neighbour combination of zhat; P half -> g_ad, R half -> g_a.
      // Summed over the warp's elements (one component per lane after the
      // first exchange) and stored per warp; k_gproj_reduce adds the slots.
      // Later exchanges write the other buffer or the spec buffers first, so
      // these reads need no barrier.
      double sr = 0.0, si = 0.0;
      if (gl) {
        const double2 xa = zb[pl.oa], xb = zb[pl.ob];
        const double xr = fma(-pl.cb, xb.x, pl.ca * xa.x);
        const double xi = fma(-pl.cb, xb.y, pl.ca * xa.y);
        if constexpr (CS) {
          // this lane's component only
          sr = (pl.r & 1) ? fma(Z.y, xr, -Z.x * xi) : fma(Z.x, xr, Z.y * xi);
        } else {
          sr = fma(Z.x, xr, Z.y * xi);
          si = fma(Z.y, xr, -Z.x * xi);
        }
      }
      if constexpr (CS) {
#pragma unroll
        for (int o = L; o < 32; o <<= 1) sr += __shfl_xor_sync(kFull, sr, o);
        // lane r < L holds the warp's sum of component r & 1 of half r >> 1;
        // store -i (sr + i si) = (si, -sr)
        const int hv = lane >> 1;
        if (lane < L && hv < 2 * Qn) {
          double* g = reinterpret_cast<double*>(gbase + ((size_t)j * Qn + (hv >> 1)) * 2 + ((hv & 1) ? 0 : 1));
          if (lane & 1)
            g[0] = sr;
          else
            g[1] = -sr;
        }
      } else if constexpr (L < 32) {
        const bool hi = lane & L;
        double k = hi ? si : sr;
        k += __shfl_xor_sync(kFull, hi ? sr : si, L);
#pragma unroll
        for (int o = 2 * L; o < 32; o <<= 1) k += __shfl_xor_sync(kFull, k, o);
        // lane r < 2Q holds sum sr of half r, lane L + r the sum si; store -i (sr + i si) = (si, -sr)
        const int r = lane & (L - 1);
        if (lane < 2 * L && r < 2 * Qn) {
          double* g = reinterpret_cast<double*>(gbase + ((size_t)j * Qn + (r >> 1)) * 2 + ((r & 1) ? 0 : 1));
          g[hi ? 0 : 1] = hi ? k : -k;
        }
      }
      // qhat^j = 2 zhat - qhat^{j+1} (+ the penalty source); within a segment
      // the next step's first iterate is already in every CTA
      if (spec) {
        cl_commit(S, pl, ahist, nxt.cc);
        ll = cl_join(pl, nxt.rn);
        qmax = nxt.qmax;
        z0 = S.zs + (size_t)((j - 1) & 1) * V;
      } else {
        double cc = 0.0;
        const double rn = cl_update<true, PEN>(pl, zh, ll, ahist, cc, psrc);
        cl_commit(S, pl, ahist, cc);
        ll = cl_join(pl, rn);
      }
      ahist = hn;
    }
  }
  stats.flush(P.status);
  cl.sync();
}

template <int QT, bool CS>
__global__ void __launch_bounds__(128, 1) k_propagate_cl(const ProbDev* __restrict__ pp, int adjoint, int j0, int j1,
                                                      double2* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const ProbDev& P = *pp;
  const int C = (int)cl.num_blocks(), crank = (int)cl.block_rank();
  const int i = blockIdx.x / C;
  const ClSmem S = cl_carve(smem, P.ncoef, P.njcoef, P.N, P.V);
  cl_setup(S, P, cl);
  const Hdr& H = *S.hdr;
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank);
  const ClAddr A = cl_addr(S, pl, C, crank);
  const ClSrc src = cl_src(P, pl, H.cq);
  double2* xv = x + (size_t)i * H.V;
  double2 rr = xv[pl.v];
  ClCount cnt;
  CtaStats stats;
  bool failed = false;
  ClHist none;
  const int n = j1 - j0;
  unsigned qmax = 0;
  if (n > 0) {
    const int rc = adjoint ? cl_start<QT, true, CS>(S, pl, A, cl_comp(pl, rr), none, false, 0.0, C, cnt, qmax)
                           : cl_start<QT, false, CS>(S, pl, A, cl_comp(pl, rr), none, false, 0.0, C, cnt, qmax);
    if (rc) {
      if (threadIdx.x == 0 && crank == 0) record_error(P.status, LB_ECUDA, adjoint ? j1 - 1 : j0);
      failed = true;
    }
  }
  const double2* z0 = S.zb + (size_t)(cnt.gk & 1) * H.V;
  ClStep nx;
  if (n > 0) nx = cl_step(src, adjoint ? j1 - 1 : j0);
  for (int jj = 0; jj < n && !failed; ++jj) {
    const int j = adjoint ? j1 - 1 - jj : j0 + jj;
    const ClStep st = nx;
    if (jj + 1 < n) nx = cl_step(src, adjoint ? j - 1 : j + 1);
    const bool spec = jj + 1 < n;
    ClNext nxt;
    double2 z;
    const int it =
        adjoint ? cl_iterate<QT, true, CS>(S, pl, A, z0, rr, st, qmax, C, cnt, z, spec, none, (jj + 1) & 1, &nxt)
                : cl_iterate<QT, false, CS>(S, pl, A, z0, rr, st, qmax, C, cnt, z, spec, none, (jj + 1) & 1, &nxt);
    if (it < 0) {
      if (threadIdx.x == 0 && crank == 0) record_error(P.status, cl_code(it), j);
      failed = true;
      break;
    }
    if (crank == 0) stats.add(adjoint ? 2 : 0, it);
    if (spec) {
      rr = cl_join(pl, nxt.rn);
      qmax = nxt.qmax;
      z0 = S.zs + (size_t)((jj + 1) & 1) * H.V;
    } else {
      double cc = 0.0;
      rr = cl_join(pl, adjoint ? cl_update<true>(pl, z, rr, none, cc) : cl_update<false>(pl, z, rr, none, cc));
    }
  }
  if (!failed && pl.ev && pl.r == 0) xv[pl.v] = rr;
  stats.flush(P.status);
  cl.sync();
}

// ---------------------------------------------------------------------------
// small kernels

// Time-independent tables: diagonal D of M and 1/(1 - dt/2 D) (Appendix A),
// digit table, coefficient tables.
__global__ void k_tables(ProbDev* __restrict__ pp) {
  const ProbDev& P = *pp;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int Q = P.Q, N = P.N;
  const double* det = P.sysp;
  const double* kerr = det + Q;
  const double* xkerr = kerr + Q;
  const double* g1 = xkerr + Q * Q;
  const double* g2 = g1 + Q;
  if (tid < N) {
    uint32_t code = 0;
    int rem = tid;
    for (int q = Q - 1; q >= 0; --q) {
      code |= (uint32_t)(rem % P.levels[q]) << (P.dbits * q);
      rem /= P.levels[q];
    }
    P.digits[tid] = code;
  }
  if (tid < P.ncoef) {
    int q = 0;
    while (q + 1 < Q && P.coff[q + 1] <= tid) ++q;
    const int n = tid - P.coff[q];
    P.cu[tid] = n + 1 < P.levels[q] ? sqrt((double)(n + 1)) : 0.0;
    P.cd[tid] = sqrt((double)n);
  }
  if (tid < P.njcoef) {
    int q = 0;
    while (q + 1 < Q && P.joff[q + 1] <= tid) ++q;
    const int r = tid - P.joff[q], n = P.levels[q];
    const int nk = r / n, nl = r % n;
    const double j = P.jump[q];
    P.jf[tid] = (nk + 1 < n && nl + 1 < n) ? j * sqrt((double)(nk + 1) * (double)(nl + 1)) : 0.0;
    P.ja[tid] = j * sqrt((double)nk * (double)nl);
  }
  if (tid < P.V) {
    const int k = tid % N, l = tid / N;
    // E_k = sum_q [delta_q n_q - xi_q/2 n_q(n_q-1)] - sum_{p<q} xi_pq n_p n_q  (H_sys, Sec. II)
    // gamma_kl = sum_q [(nk - nl)^2/(2 T2) + (nk + nl)/(2 T1)]                 (collapse operators)
    int dk[LB_MAXQ], dl[LB_MAXQ];
    int rk = k, rl = l;
    for (int q = Q - 1; q >= 0; --q) {
      dk[q] = rk % P.levels[q];
      rk /= P.levels[q];
      dl[q] = rl % P.levels[q];
      rl /= P.levels[q];
    }
    double Ek = 0.0, El = 0.0, gam = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double a = dk[q], b = dl[q];
      Ek += det[q] * a - 0.5 * kerr[q] * a * (a - 1.0);
      El += det[q] * b - 0.5 * kerr[q] * b * (b - 1.0);
      gam += 0.5 * (a - b) * (a - b) * g2[q] + 0.5 * (a + b) * g1[q];
      for (int p = 0; p < q; ++p) {
        Ek -= xkerr[p * Q + q] * dk[p] * a;
        El -= xkerr[p * Q + q] * dl[p] * b;
      }
    }
    const double2 D = make_double2(-gam, -(Ek - El));  // -i(E_k - E_l) - gamma_kl
    P.D[tid] = D;
    const double hh = 0.5 * P.h;
    const double ar = 1.0 - hh * D.x, ai = -hh * D.y;  // 1 - dt/2 D
    const double den = ar * ar + ai * ai;
    P.Dinv[tid] = make_double2(ar / den, -ai / den);
  }
}

// rho_i^tar = V rho_i(0) V^+ with V lifted to the full space (Sec. III-C)
__global__ void k_gate_targets(ProbDev P, const double2* __restrict__ Vg, const int32_t* __restrict__ emap,
                               const int32_t* __restrict__ efull, int Ne) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)P.M * P.V) return;
  const int i = (int)(tid / P.V), v = (int)(tid % P.V);
  const int k = v % P.N, l = v / P.N;
  const int ek = emap[k], el = emap[l];
  double2 acc = make_double2(0.0, 0.0);
  if (ek >= 0 && el >= 0) {
    const double2* r = P.q0 + (size_t)i * P.V;
    for (int b = 0; b < Ne; ++b) {
      const double2 vb = Vg[el + (size_t)Ne * b];  // V[el, b]
      for (int a = 0; a < Ne; ++a) {
        const double2 va = Vg[ek + (size_t)Ne * a];  // V[ek, a]
        const double2 x = r[efull[a] + (size_t)P.N * efull[b]];
        // va * x * conj(vb)
        const double tr = va.x * x.x - va.y * x.y, ti = va.x * x.y + va.y * x.x;
        acc.x += tr * vb.x + ti * vb.y;
        acc.y += ti * vb.x - tr * vb.y;
      }
    }
  }
  P.tar[tid] = acc;
}

// (dt/2) d_q(t_j + dt/2) for every step j and subsystem q (eq. rotctrl)
__global__ void k_control_table(const ProbDev* __restrict__ pp) {
  const ProbDev& P = *pp;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)P.NT * P.cq) return;
  const int j = (int)(tid / P.cq), q = (int)(tid % P.cq);
  const double t = (j + 0.5) * P.h;
  if (q >= P.Q) {
    // Jaynes-Cummings pair: (dt/2) g e^{i eta t}
    const int k = q - P.Q;
    double sn, cs;
    sincos(P.je[k] * t, &sn, &cs);
    const double gg = 0.5 * P.h * P.jg[k];
    P.ctab[tid] = make_double2(gg * cs, gg * sn);
    return;
  }
  const double dtau = P.T / (P.Ns - 2);
  const double x = t / dtau;
  const int slo = max(0, (int)floor(x - 1.0)), shi = min(P.Ns - 1, (int)floor(x + 2.0));
  double dr = 0.0, di = 0.0;
  for (int f = 0; f < P.nf[q]; ++f) {
    double sn, cs;
    sincos(P.carriers[P.foff[q] + f] * t, &sn, &cs);
    double wr = 0.0, wi = 0.0;
    for (int s = slo; s <= shi; ++s) {
      const double S = bspline2(x - (s - 0.5));
      const double* a = P.alpha + P.aoff[q] + 2 * (f * P.Ns + s);
      wr += S * a[0];
      wi += S * a[1];
    }
    dr += wr * cs - wi * sn;
    di += wr * sn + wi * cs;
  }
  const double sc = 0.5 * P.h * kTwoPi;
  P.ctab[tid] = make_double2(sc * dr, sc * di);
}

// rho_j >= ||(I - dt/2 D)^-1 dt/2 O_j||_inf and the same for the adjoint:
// |(I - dt/2 D)^-1| <= 1 (Re D <= 0); per subsystem the control couplings of
// one row (or column) sum to at most |dt/2 d_q| 2 (sqrt(n-1) + sqrt(n-2)), and
// the decay sandwich to at most (dt/2)/T1 (n - 1).  One thread per step.
__global__ void k_stop_factors(const ProbDev* __restrict__ pp) {
  const ProbDev& P = *pp;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= P.NT) return;
  double rho = 0.0;
  for (int q = 0; q < P.Q; ++q) {
    const double n = P.levels[q];
    const double2 c = P.ctab[(size_t)j * P.cq + q];
    rho += hypot(c.x, c.y) * 2.0 * (sqrt(n - 1.0) + sqrt(n - 2.0)) + P.jump[q] * (n - 1.0);
  }
  // each of the four terms of a Jaynes-Cummings pair couples with at most
  // |dt/2 g| sqrt((n_p - 1)(n_q - 1))
  for (int k = 0; k < P.npair; ++k) {
    const double2 c = P.ctab[(size_t)j * P.cq + P.Q + k];
    rho += 4.0 * hypot(c.x, c.y) * sqrt((P.levels[P.jp[k]] - 1.0) * (P.levels[P.jq[k]] - 1.0));
  }
  // (1 - rho)/rho, capped so that rtol ||q|| times it stays finite
  P.sfac[j] = rho < 0.5 ? fmin((1.0 - rho) / fmax(rho, 1e-200), 1e200) : 1.0;
  // running penalty weight dt beta(t_j), beta(t) = exp(-((t - T)/a)^2)/a, left rectangle rule
  if (P.gamma1 != 0.0) {
    const double x = (j * P.h - P.T) / P.pen_a;
    P.pen[j] = P.h * exp(-x * x) / P.pen_a;
  }
}

// G = sum_i beta_i/M J_i + gamma2/2 ||alpha||^2 (eq. optimproblem), one warp
__global__ void k_objective(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.x];
  const int lane = threadIdx.x;
  double s = 0.0, a2 = 0.0;
  for (int i = lane; i < P.M; i += 32) s += P.wgt[i] * P.J[i];
  for (int k = lane; k < P.n_params; k += 32) a2 += P.alpha[k] * P.alpha[k];
  s = warp_sum(s);
  a2 = warp_sum(a2);
  if (lane == 0) P.G[0] = s + 0.5 * P.gamma2 * a2;
}

// Sum of the gradient pieces over their gM state slots (states, CTAs, warps),
// in slot order, for every (step, subsystem, piece): gsum[NT][Q][2].
__global__ void k_gproj_reduce(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const size_t n = (size_t)P.NT * P.Q * 2, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    double2 t = make_double2(0.0, 0.0);
    for (int i = 0; i < P.gM; ++i) {
      const double2 g = P.gproj[(size_t)i * n + k];
      t.x += g.x;
      t.y += g.y;
    }
    P.gsum[k] = t;
  }
}

// dG/dalpha (eq. reducedgradient): one warp per (q, f, s); the sum over the
// spline's support in time is in a fixed order (the states were summed by
// k_gproj_reduce).
__global__ void k_gradient_project(const ProbDev* __restrict__ probs) {
  const ProbDev& P = probs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int q = 0, rem = gw;
  while (q < P.Q && rem >= P.nf[q] * P.Ns) {
    rem -= P.nf[q] * P.Ns;
    ++q;
  }
  if (q >= P.Q) return;
  const int f = rem / P.Ns, s = rem % P.Ns;
  const double om = P.carriers[P.foff[q] + f];
  const double dtau = P.T / (P.Ns - 2);
  // S_s(t) > 0 for t in ((s - 2) dtau, (s + 1) dtau)
  const int jlo = max(0, (int)floor((s - 2) * dtau / P.h - 1.0));
  const int jhi = min(P.NT - 1, (int)ceil((s + 1) * dtau / P.h));
  double gr = 0.0, gi = 0.0;
  for (int j = jlo + lane; j <= jhi; j += 32) {
    const double t = (j + 0.5) * P.h;
    const double S = bspline2(t / dtau - (s - 0.5));
    if (S == 0.0) continue;
    const double2* g = P.gsum + ((size_t)j * P.Q + q) * 2;
    const double ga_r = g[0].x, ga_i = g[0].y, gd_r = g[1].x, gd_i = g[1].y;
    double sn, cs;
    sincos(om * t, &sn, &cs);
    // Re(e^{iOt} g_a + e^{-iOt} g_ad) and Re(i e^{iOt} g_a - i e^{-iOt} g_ad)
    gr += S * (cs * ga_r - sn * ga_i + cs * gd_r + sn * gd_i);
    gi += S * (-(cs * ga_i + sn * ga_r) + cs * gd_i - sn * gd_r);
  }
  gr = warp_sum(gr);
  gi = warp_sum(gi);
  if (lane == 0) {
    const int k = P.aoff[q] + 2 * (f * P.Ns + s);
    const double sc = P.h * kTwoPi;
    P.grad[k] = sc * gr + P.gamma2 * P.alpha[k];
    P.grad[k + 1] = sc * gi + P.gamma2 * P.alpha[k + 1];
  }
}

// G, gradient and status of every system of a batch into contiguous arrays
__global__ void k_gather(const ProbDev* __restrict__ probs, const int64_t* __restrict__ grad_off,
                         double* __restrict__ G_all, double* __restrict__ grad_all, DevStatus* __restrict__ st_all) {
  const ProbDev& P = probs[blockIdx.x];
  if (threadIdx.x == 0) {
    if (G_all) G_all[blockIdx.x] = P.G[0];
    if (st_all) st_all[blockIdx.x] = *P.status;
  }
  if (grad_all)
    for (int k = threadIdx.x; k < P.n_params; k += blockDim.x) grad_all[grad_off[blockIdx.x] + k] = P.grad[k];
}

// y = M^{j+1/2} x or (M^{j+1/2})^+ x, one thread per element
template <bool ADJ>
__global__ void k_apply(const ProbDev* __restrict__ pp, int step, const double2* __restrict__ x,
                        double2* __restrict__ y, int n_vec) {
  __shared__ Hdr H;
  const ProbDev& P = *pp;
  if (threadIdx.x == 0) load_hdr(H, P);
  __syncthreads();
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (size_t)n_vec * H.V) return;
  const int b = (int)(tid / H.V), v = (int)(tid % H.V);
  const int k = v % H.N, l = v / H.N;
  const Tabs T{P.cu, P.cd, P.jf, P.ja};
  const double2* xv = x + (size_t)b * H.V;
  double ar = 0.0, ai = 0.0;
  offdiag_acc<ADJ>(ar, ai, xv, v, P.digits[k], P.digits[l], H, T, P.ctab + (size_t)step * H.cq);
  const double inv = 2.0 / H.h;
  const double2 D = P.D[v];
  const double di = ADJ ? -D.y : D.y;
  const double2 xx = xv[v];
  y[tid] = make_double2(fma(D.x, xx.x, -di * xx.y) + inv * ar, fma(D.x, xx.y, di * xx.x) + inv * ai);
}


// ---------------------------------------------------------------------------
// grid-wide persistent sweeps (states too large for one CTA's shared memory)
//
// One cooperative launch keeps every SM busy on all M states at once.  Block
// b owns a contiguous chunk of the flattened [M][V] element range; each inner
// iteration reads the previous iterate of every element (neighbours through
// L2, bypassing L1) and ends with a grid barrier.  Per-state maxima of
// |z_new - z| and |q| are combined with atomicMax on the integer bit patterns
// (order independent), so every block takes the same stopping decision and a
// recompute is bit-identical.

constexpr long long kSpinLimit = 1LL << 26;  // ~seconds of polling before a barrier gives up

// Grid barrier with a bounded wait.  Returns false on every block once a
// wait has given up (the kernel then returns).
__device__ bool grid_sync(GridBar* bar, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    volatile int* verr = &bar->err;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    int ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (*verr) {
          ok = 0;
          break;
        }
        __nanosleep(64);
        if (++spins > kSpinLimit) {
          atomicExch(&bar->err, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (*verr) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct GridHdr {
  Hdr h;
  int M;
  int herm;         // Hermitian symmetry: only elements k <= l are iterated, the rest mirrored
  int Vh;           // elements per state in the loops: V, or N (N + 1) / 2 with herm
  long long total;  // M * Vh
  long long chunk;  // elements per block
};

// Element e of a grid sweep's loops: state b and vec index v; with the
// Hermitian symmetry the loops visit k <= l only (v from the table hmap) and
// vm is the mirror index l + N k of an off-diagonal element, whose value is
// the conjugate (-1 for diagonal elements and without the symmetry).
struct GEl {
  int b, v, vm;
};
__device__ __forceinline__ GEl gel(const GridHdr& G, const int32_t* __restrict__ hmap, long long e) {
  GEl r;
  if (!G.herm) {
    r.b = (int)(e / G.h.V);
    r.v = (int)(e - (long long)r.b * G.h.V);
    r.vm = -1;
    return r;
  }
  r.b = (int)(e / G.Vh);
  r.v = __ldg(hmap + (e - (long long)r.b * G.Vh));
  const int N = G.h.N, k = r.v % N, l = r.v / N;
  r.vm = k != l ? l + N * k : -1;
  return r;
}
// store x at element g of the state array a (and its mirror)
__device__ __forceinline__ void gput(double2* a, const GEl& g, int V, double2 x) {
  a[(size_t)g.b * V + g.v] = x;
  if (g.vm >= 0) a[(size_t)g.b * V + g.vm] = make_double2(x.x, -x.y);
}

__host__ __device__ inline size_t grid_smem_bytes_impl(int ncoef, int njcoef) {
  return align16(sizeof(GridHdr)) + align16(sizeof(double) * 2 * ncoef) + align16(sizeof(double) * 2 * njcoef) +
         align16(sizeof(double) * 4 * 8) + 64;
}

struct GridSmem {
  GridHdr* g;
  double* cu;
  double* cd;
  double* jf;
  double* ja;
  double* red;  // [4][8 warps]
  int* flag;
};

__device__ GridSmem grid_setup(unsigned char* base, const ProbDev& P, int nstates, int herm) {
  GridSmem S;
  size_t o = 0;
  S.g = reinterpret_cast<GridHdr*>(base + o);
  o += align16(sizeof(GridHdr));
  S.cu = reinterpret_cast<double*>(base + o);
  S.cd = S.cu + P.ncoef;
  o += align16(sizeof(double) * 2 * P.ncoef);
  S.jf = reinterpret_cast<double*>(base + o);
  S.ja = S.jf + P.njcoef;
  o += align16(sizeof(double) * 2 * P.njcoef);
  S.red = reinterpret_cast<double*>(base + o);
  o += align16(sizeof(double) * 4 * 8);
  S.flag = reinterpret_cast<int*>(base + o);
  if (threadIdx.x == 0) {
    load_hdr(S.g->h, P);
    S.g->M = nstates;
    S.g->herm = herm;
    S.g->Vh = herm ? P.N * (P.N + 1) / 2 : P.V;
    S.g->total = (long long)nstates * S.g->Vh;
    const long long per = (S.g->total + gridDim.x - 1) / gridDim.x;
    // whole warps, not whole blocks: rounding the chunk up to the block size
    // left up to half of the blocks without elements (three states of
    // N (N + 1) / 2 = 32896 elements filled 193 of 304 blocks)
    S.g->chunk = (per + 31) / 32 * 32;
  }
  for (int i = threadIdx.x; i < P.ncoef; i += blockDim.x) {
    S.cu[i] = P.cu[i];
    S.cd[i] = P.cd[i];
  }
  for (int i = threadIdx.x; i < P.njcoef; i += blockDim.x) {
    S.jf[i] = P.jf[i];
    S.ja[i] = P.ja[i];
  }
  __syncthreads();
  return S;
}

// Flush a per-thread running maximum for state b into the global slot.
__device__ __forceinline__ void flush_max(unsigned long long* slots, int b, unsigned long long m) {
  if (b >= 0 && m) atomicMax(slots + b, m);
}

// Per-state maxima over a block's chunk [e0, e1).  When the chunk covers at
// most kLocalStates states (large states), each thread keeps one maximum per
// state in registers and the block pushes one atomicMax per state; otherwise
// (many small states per block) each thread pushes its own running maximum.
// `local` depends only on the chunk, so it is uniform over the block.
constexpr int kLocalStates = 4;

struct StateMax {
  int sb0, ns;
  bool local;
  unsigned long long m[kLocalStates];
  int bcur;
  unsigned long long mcur;

  __device__ void init(long long e0, long long e1, int V) {
    sb0 = (int)(e0 / V);
    const int sb1 = e1 > e0 ? (int)((e1 - 1) / V) : sb0;
    ns = sb1 - sb0 + 1;
    local = ns <= kLocalStates;
#pragma unroll
    for (int k = 0; k < kLocalStates; ++k) m[k] = 0;
    bcur = -1;
    mcur = 0;
  }
  __device__ __forceinline__ void add(int b, unsigned long long x, unsigned long long* slots) {
    if (local) {
      const int i = b - sb0;
#pragma unroll
      for (int k = 0; k < kLocalStates; ++k)
        if (k == i) m[k] = umax64(m[k], x);
    } else {
      if (b != bcur) {
        flush_max(slots, bcur, mcur);
        bcur = b;
        mcur = 0;
      }
      mcur = umax64(mcur, x);
    }
  }
  // all threads of the block call this
  __device__ void push(unsigned long long* slots, unsigned long long* red) {
    if (local) {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
      for (int k = 0; k < kLocalStates; ++k) {
        const unsigned long long v = warp_max_u64(m[k]);
        if (lane == 0) red[k * 8 + warp] = v;
      }
      __syncthreads();
      if ((int)threadIdx.x < ns) {
        unsigned long long r = 0;
        for (int w = 0; w < nwarps; ++w) r = umax64(r, red[threadIdx.x * 8 + w]);
        if (r) atomicMax(slots + sb0 + threadIdx.x, r);
      }
      __syncthreads();
    } else {
      flush_max(slots, bcur, mcur);
    }
  }
};

// One implicit-midpoint solve over all M states: z satisfies
// (I - dt/2 M) z = rhs (ADJ: M^+) to the per-state tolerance.  `it_global`
// counts iterations and `solve` counts solves across the launch; they select
// the banks of the per-state maxima.  Returns the iteration count, -1
// (max_iter), -2 (NaN/Inf) or -3 (a barrier wait gave up); on success *zout
// points at the buffer holding z.
// First-iterate predictor of the grid sweeps: the off-diagonal corrections
// c = (I - dt/2 D) z - rhs of the last n steps, kept per element in the ring
// P.hist (each element always handled by the same thread, so no
// synchronisation is needed), extrapolated as in the cluster sweeps.
struct GridHist {
  int n = 0, slot = 0;
  __device__ void advance() {
    n = n < kPredOrder ? n + 1 : kPredOrder;
    slot = slot + 1 < kPredOrder ? slot + 1 : 0;
  }
};

template <bool ADJ>
__device__ __forceinline__ void grid_record(const ProbDev& P, size_t stride, GridHist h, size_t o, int v,
                                            double hh, double2 z, double2 r) {
  const double2 D = __ldg(P.D + v);
  const double dr = hh * D.x, di = hh * (ADJ ? -D.y : D.y);
  const double cr = z.x - fma(dr, z.x, -di * z.y) - r.x;
  const double ci = z.y - fma(dr, z.y, di * z.x) - r.y;
  P.hist[(size_t)h.slot * stride + o] = make_double2(cr, ci);
}

template <bool ADJ>
__device__ int grid_solve(const ProbDev& P, const GridSmem& S, const double2* __restrict__ rhs,
                          const double2* __restrict__ ct, double fac, long long& it_global, long long& solve,
                          double2** zout, GridHist hist = GridHist()) {
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  const bool neumann = H.method == LB_SOLVER_NEUMANN;
  const int M = G.M, V = H.V, N = H.N;
  const long long e0 = (long long)blockIdx.x * G.chunk;
  const long long e1 = min(G.total, e0 + G.chunk);
  unsigned long long* dslots = P.gslots;          // [3][M]
  unsigned long long* qslots = P.gslots + 3 * M;  // [2][M]
  unsigned long long* qbank = qslots + (solve & 1) * M;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(S.red);
  // z_0 = (I - dt/2 D)^-1 rhs (Jacobi) or rhs (Neumann); per-state max |rhs|
  {
    StateMax sm;
    sm.init(e0, e1, G.Vh);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const GEl g = gel(G, P.hmap, e);
      const int b = g.b, v = g.v;
      const size_t o = (size_t)b * V + v;
      const double2 r = rhs[o];
      double2 z0 = r;
      if (!neumann) {
        double ur = r.x, ui = r.y;
        int sl = hist.slot;
        for (int i = 1; i <= hist.n; ++i) {
          sl = sl > 0 ? sl - 1 : kPredOrder - 1;
          const double w = kExtrap[hist.n][i - 1];
          const double2 c = P.hist[(size_t)sl * ((size_t)M * V) + o];
          ur = fma(w, c.x, ur);
          ui = fma(w, c.y, ui);
        }
        const double2 d = __ldg(P.Dinv + v);
        const double di = ADJ ? -d.y : d.y;
        z0 = make_double2(fma(d.x, ur, -di * ui), fma(d.x, ui, di * ur));
      }
      gput(P.zA, g, V, z0);
      sm.add(b, umax64(abs_bits(r.x), abs_bits(r.y)), qbank);
    }
    sm.push(qbank, red);
  }
  if (!grid_sync(P.bar, gridDim.x)) return -3;
  // the previous solve's |q| bank is free again: clear it for the next solve
  if (blockIdx.x == 0)
    for (int b = threadIdx.x; b < M; b += blockDim.x) qslots[((solve + 1) & 1) * M + b] = 0;
  ++solve;
  const double hh = 0.5 * H.h;
  double2* zc = P.zA;
  double2* zn = P.zB;
  for (int it = 0; it < H.max_iter; ++it, ++it_global) {
    unsigned long long* bank = dslots + (it_global % 3) * M;
    StateMax sm;
    sm.init(e0, e1, G.Vh);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const GEl g = gel(G, P.hmap, e);
      const int b = g.b, v = g.v;
      const double2* xs = zc + (size_t)b * V;
      const int k = v % N, l = v / N;
      const double2 r = rhs[(size_t)b * V + v];
      double ar = r.x, ai = r.y;
      offdiag_acc<ADJ, true>(ar, ai, xs, v, __ldg(P.digits + k), __ldg(P.digits + l), H, T, ct);
      const double2 zo = __ldcg(xs + v);
      double2 z;
      if (!neumann) {
        const double2 d = __ldg(P.Dinv + v);
        const double di = ADJ ? -d.y : d.y;
        z.x = fma(d.x, ar, -di * ai);
        z.y = fma(d.x, ai, di * ar);
      } else {
        const double2 D = __ldg(P.D + v);
        const double dr = hh * D.x, di = hh * (ADJ ? -D.y : D.y);
        z.x = ar + fma(dr, zo.x, -di * zo.y);
        z.y = ai + fma(dr, zo.y, di * zo.x);
      }
      gput(zn, g, V, z);
      sm.add(b, umax64(abs_bits(z.x - zo.x), abs_bits(z.y - zo.y)), bank);
    }
    sm.push(bank, red);
    if (!grid_sync(P.bar, gridDim.x)) return -3;
    // bank of iteration it_global + 2 is no longer read by anyone: clear it
    if (blockIdx.x == 0)
      for (int b = threadIdx.x; b < M; b += blockDim.x) dslots[((it_global + 2) % 3) * M + b] = 0;
    // every block takes the same decision from the same slots
    if (threadIdx.x == 0) {
      int state = 1;  // 1 converged, 0 not yet, -2 NaN/Inf
      for (int b = 0; b < M; ++b) {
        const unsigned long long d = __ldcg(bank + b);
        const unsigned long long q = __ldcg(qbank + b);
        if (d >= kInfBits || q >= kInfBits) {
          state = -2;
          break;
        }
        const unsigned long long thr = abs_bits(H.rtol * __longlong_as_double((long long)q) * fac);
        if (d > thr) state = 0;
      }
      *S.flag = state;
    }
    __syncthreads();
    const int state = *S.flag;
    __syncthreads();
    double2* t = zc;
    zc = zn;
    zn = t;
    if (state == -2) return -2;
    if (state == 1) {
      ++it_global;
      *zout = zc;
      return it + 1;
    }
  }
  return -1;
}

__device__ void grid_fail(const ProbDev& P, int code, int step) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    record_error(P.status, code == -1 ? LB_ENOTCONV : (code == -2 ? LB_ENAN : LB_ECUDA), step);
}

// mode 0: forward sweep on P.qT (from P.q0 if init), checkpoints if tape
// mode 1: forward steps j0..j1-1 in place on x; mode 2: adjoint steps j1-1..j0 in place on x
__global__ void __launch_bounds__(kGridThreads, 2) k_sweep_grid(const ProbDev* __restrict__ pp, int mode, int init,
                                                             int tape, int j0, int j1, double2* __restrict__ x,
                                                             int nstates) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ProbDev& P = *pp;
  // the Hermitian symmetry only for the forward sweep over the system's own
  // states (vectors given to lb_propagate may be anything)
  const GridSmem S = grid_setup(smem, P, mode == 0 ? P.M : nstates, mode == 0 ? P.herm : 0);
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const int V = H.V;
  double2* q = mode == 0 ? P.qT : x;
  const long long e0 = (long long)blockIdx.x * G.chunk, e1 = min(G.total, e0 + G.chunk);
  const size_t hstride = (size_t)G.M * V;
  if (mode == 0 && init)
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const GEl g = gel(G, P.hmap, e);
      gput(q, g, V, P.q0[(size_t)g.b * V + g.v]);
    }
  long long itg = 0, nsolve = 0;
  unsigned long long iters = 0, steps = 0;
  int maxit = 0;
  const int phase = mode == 2 ? 2 : 0;
  // predictor only when no step is ever recomputed (K == 0), as in the other sweeps
  const bool pred = mode == 0 && H.K == 0 && H.method != LB_SOLVER_NEUMANN;
  const double hh = 0.5 * H.h;
  GridHist hist;
  for (int jj = 0; jj < j1 - j0; ++jj) {
    const int j = mode == 2 ? j1 - 1 - jj : j0 + jj;
    if (mode == 0 && tape && H.K > 0 && j % H.K == 0) {
      for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const GEl g = gel(G, P.hmap, e);
        const double2 qq = q[(size_t)g.b * V + g.v];
        gput(P.ckpt + ((size_t)g.b * H.n_ckpt + j / H.K) * V, GEl{0, g.v, g.vm}, V, qq);
      }
    }
    double2* z = nullptr;
    const int it = mode == 2 ? grid_solve<true>(P, S, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve, &z)
                             : grid_solve<false>(P, S, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve, &z,
                                                 pred ? hist : GridHist());
    if (it < 0) {
      grid_fail(P, it, j);
      break;
    }
    iters += (unsigned long long)it * G.M;
    steps += G.M;
    maxit = max(maxit, it);
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const GEl g = gel(G, P.hmap, e);
      const size_t o = (size_t)g.b * V + g.v;
      const double2 zz = z[o], qq = q[o];
      if (mode == 0 && tape && H.K == 0) gput(P.ckpt + ((size_t)g.b * H.NT + j) * V, GEl{0, g.v, g.vm}, V, zz);
      if (pred) grid_record<false>(P, hstride, hist, o, g.v, hh, zz, qq);
      gput(q, g, V, make_double2(fma(2.0, zz.x, -qq.x), fma(2.0, zz.y, -qq.y)));
    }
    if (pred) hist.advance();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&P.status->iters[phase], iters);
    atomicAdd(&P.status->steps[phase], steps);
    atomicMax(&P.status->max_iter_seen, maxit);
  }
}

// backward sweep over all states: recompute each checkpoint segment, then the
// adjoint steps with the gradient pieces summed over states and blocks
__global__ void __launch_bounds__(kGridThreads, 2) k_backward_grid(const ProbDev* __restrict__ pp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ProbDev& P = *pp;
  const GridSmem S = grid_setup(smem, P, P.M, P.herm);
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const int V = H.V, N = H.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const long long e0 = (long long)blockIdx.x * G.chunk, e1 = min(G.total, e0 + G.chunk);
  const size_t hstride = (size_t)G.M * V;
  // terminal condition qhat^{N_T} = beta_i/M g_i (Appendix B)
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const GEl g = gel(G, P.hmap, e);
    const size_t o = (size_t)g.b * V + g.v;
    const double w = P.wgt[g.b];
    const double wt = linear_sign(P.kind) * w;
    const double2 t = P.tar[o];
    if (H.kind == LB_J_FROB) {
      const double2 qq = P.qT[o];
      gput(P.lam, g, V, make_double2(w * (qq.x - t.x), w * (qq.y - t.y)));
    } else {
      gput(P.lam, g, V, make_double2(wt * t.x, wt * t.y));
    }
  }
  long long itg = 0, nsolve = 0;
  unsigned long long it_rec = 0, st_rec = 0, it_adj = 0, st_adj = 0;
  int maxit = 0;
  const int nseg = H.K > 0 ? (H.NT + H.K - 1) / H.K : 1;
  bool failed = false;
  // adjoint predictor: the adjoint steps come in the same order for every K
  const bool apred = H.method != LB_SOLVER_NEUMANN;
  const double hh = 0.5 * H.h;
  GridHist ahist;
  for (int sg = nseg - 1; sg >= 0 && !failed; --sg) {
    const int j0 = H.K > 0 ? sg * H.K : 0;
    const int j1 = H.K > 0 ? min(H.NT, j0 + H.K) : H.NT;
    if (H.K > 0) {
      for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const GEl g = gel(G, P.hmap, e);
        gput(P.qf, g, V, P.ckpt[((size_t)g.b * H.n_ckpt + sg) * V + g.v]);
      }
      for (int j = j0; j < j1; ++j) {
        double2* z = nullptr;
        const int it = grid_solve<false>(P, S, P.qf, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve, &z);
        if (it < 0) {
          grid_fail(P, it, j);
          failed = true;
          break;
        }
        it_rec += (unsigned long long)it * G.M;
        st_rec += G.M;
        maxit = max(maxit, it);
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          const GEl g = gel(G, P.hmap, e);
          const size_t o = (size_t)g.b * V + g.v;
          const double2 zz = z[o], qq = P.qf[o];
          P.seg[((size_t)g.b * H.K + (j - j0)) * V + g.v] = zz;  // read back at the same element only
          gput(P.qf, g, V, make_double2(fma(2.0, zz.x, -qq.x), fma(2.0, zz.y, -qq.y)));
        }
      }
      if (failed) break;
    }
    for (int j = j1 - 1; j >= j0; --j) {
      const double2* ct = P.ctab + (size_t)j * H.cq;
      double2* zh = nullptr;
      const int it = grid_solve<true>(P, S, P.lam, ct, stop_factor(P, j), itg, nsolve, &zh, apred ? ahist : GridHist());
      if (it < 0) {
        grid_fail(P, it, j);
        failed = true;
        break;
      }
      it_adj += (unsigned long long)it * G.M;
      st_adj += G.M;
      maxit = max(maxit, it);
      // gradient pieces (eq. reducedgradient), summed over this block's elements
      for (int q = 0; q < H.Q; ++q) {
        const int n = H.lev[q], s = H.stride[q], co = H.coff[q], sN = s * N;
        double sar = 0.0, sai = 0.0, sdr = 0.0, sdi = 0.0;
        for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
          const GEl g = gel(G, P.hmap, e);
          const int b = g.b, v = g.v;
          const double2* zs = zh + (size_t)b * V;
          const double2 Z = H.K > 0 ? P.seg[((size_t)b * H.K + (j - j0)) * V + v]
                                    : P.ckpt[((size_t)b * H.NT + j) * V + v];
          const int k = v % N, l = v / N;
          const uint32_t kd = __ldg(P.digits + k), ld = __ldg(P.digits + l);
          const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
          const double c1 = S.cu[co + nk], c2 = S.cd[co + nl], c3 = S.cd[co + nk], c4 = S.cu[co + nl];
          const double2 x1 = __ldcg(zs + v + (nk + 1 < n ? s : 0));
          const double2 x2 = __ldcg(zs + v - (nl > 0 ? sN : 0));
          const double2 x3 = __ldcg(zs + v - (nk > 0 ? s : 0));
          const double2 x4 = __ldcg(zs + v + (nl + 1 < n ? sN : 0));
          const double pr = fma(-c2, x2.x, c1 * x1.x);
          const double pi = fma(-c2, x2.y, c1 * x1.y);
          const double rr = fma(-c4, x4.x, c3 * x3.x);
          const double ri = fma(-c4, x4.y, c3 * x3.y);
          if (g.vm < 0) {
            sar = fma(Z.x, rr, fma(Z.y, ri, sar));
            sai = fma(Z.y, rr, fma(-Z.x, ri, sai));
            sdr = fma(Z.x, pr, fma(Z.y, pi, sdr));
            sdi = fma(Z.y, pr, fma(-Z.x, pi, sdi));
          } else {
            // Hermitian Z and zhat: the mirror element (l, k) adds -conj(B) to
            // the g_a sum and -conj(A) to the g_ad sum, A = Z conj(R), B = Z conj(P)
            const double ar = fma(Z.x, rr, Z.y * ri), ai = fma(Z.y, rr, -Z.x * ri);
            const double br = fma(Z.x, pr, Z.y * pi), bi = fma(Z.y, pr, -Z.x * pi);
            sar += ar - br;
            sai += ai + bi;
            sdr += br - ar;
            sdi += bi + ai;
          }
        }
        const double r = warp_sum4(sar, sai, sdr, sdi, lane);
        if ((lane & 7) == 0) S.red[(lane >> 3) * 8 + warp] = r;
        __syncthreads();
        if (threadIdx.x < 4) {
          double t = 0.0;
          for (int w = 0; w < nwarps; ++w) t += S.red[threadIdx.x * 8 + w];
          P.partials[((size_t)blockIdx.x * LB_MAXQ + q) * 4 + threadIdx.x] = t;
        }
        __syncthreads();
      }
      // qhat^j = 2 zhat - qhat^{j+1}
      for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const GEl g = gel(G, P.hmap, e);
        const size_t o = (size_t)g.b * V + g.v;
        const double2 z = zh[o], ll = P.lam[o];
        if (apred) grid_record<true>(P, hstride, ahist, o, g.v, hh, z, ll);
        gput(P.lam, g, V, make_double2(fma(2.0, z.x, -ll.x), fma(2.0, z.y, -ll.y)));
      }
      if (apred) ahist.advance();
      if (!grid_sync(P.bar, gridDim.x)) {
        grid_fail(P, -3, j);
        failed = true;
        break;
      }
      // block 0: fixed-order sum over blocks; multiply by -i: g = (S.im, -S.re)
      if (blockIdx.x == 0 && threadIdx.x < 4 * H.Q) {
        const int q = threadIdx.x >> 2, c = threadIdx.x & 3;
        double t = 0.0;
        for (int bb = 0; bb < (int)gridDim.x; ++bb) t += P.partials[((size_t)bb * LB_MAXQ + q) * 4 + c];
        double* g = reinterpret_cast<double*>(P.gproj + ((size_t)j * H.Q + q) * 2);
        if (c == 0) g[1] = -t;
        if (c == 1) g[0] = t;
        if (c == 2) g[3] = -t;
        if (c == 3) g[2] = t;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&P.status->iters[1], it_rec);
    atomicAdd(&P.status->steps[1], st_rec);
    atomicAdd(&P.status->iters[2], it_adj);
    atomicAdd(&P.status->steps[2], st_adj);
    atomicMax(&P.status->max_iter_seen, maxit);
  }
}

// J_i per state from P.qT (one block per state, fixed-order reduction)
__global__ void k_objective_states(const ProbDev* __restrict__ pp) {
  const ProbDev& P = *pp;
  __shared__ double red[32];
  const int i = blockIdx.x;
  const size_t base = (size_t)i * P.V;
  double acc = 0.0;
  for (int v = threadIdx.x; v < P.V; v += blockDim.x) {
    const double2 q = P.qT[base + v];
    const double2 t = P.tar[base + v];
    if (P.kind == LB_J_FROB) {
      const double dr = q.x - t.x, di = q.y - t.y;
      acc = fma(dr, dr, fma(di, di, acc));
    } else {
      acc = fma(t.x, q.x, fma(t.y, q.y, acc));
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    P.J[i] = merit_value(P.kind, t);
  }
}
}  // namespace

// ---------------------------------------------------------------------------
// launchers

int gmres_krylov_dim(int V, int ncoef, int njcoef, int N, size_t smem_limit) {
  const size_t base = res_smem_bytes(ncoef, njcoef, N, V, 1) - sizeof(double2);
  if (base >= smem_limit) return 0;
  long long m = (long long)((smem_limit - base) / (sizeof(double2) * (size_t)V)) - 1;
  if (m > kGmresMaxM) m = kGmresMaxM;
  return m >= kGmresMinM ? (int)m : 0;
}

ResidentConfig resident_config(int maxV, int maxQ, int maxNcoef, int maxNj, int maxN, bool uniformQ,
                               size_t kry_elems) {
  ResidentConfig rc;
  int E = 1;
  while (E < 8 && (maxV + E - 1) / E > 512) E *= 2;
  int threads = (maxV + E - 1) / E;
  threads = ((threads + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  rc.threads = threads;
  rc.E = E;
  rc.QT = (E == 1 && uniformQ && maxQ <= 4) ? maxQ : 0;
  rc.smem = res_smem_bytes(maxNcoef, maxNj, maxN, maxV, kry_elems);
  rc.gmres = kry_elems > 0;
  return rc;
}

template <int E, int QT, bool GM>
static cudaError_t set_smem_attr(size_t smem) {
  cudaError_t e =
      cudaFuncSetAttribute(k_forward_res<E, QT, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_backward_res<E, QT, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_propagate_res<E, QT, GM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Kernel instantiations: element count per thread E, for E == 1 the
// compile-time subsystem count QT of the per-thread plan (0 = generic path),
// and GM for the variants that can run GMRES (generic path only).
template <int E, int QT, bool GM = false>
struct ResKernels {
  static cudaError_t fwd(dim3 g, dim3 b, size_t sm, cudaStream_t s, const ProbDev* p, const WorkItem* it, int tape) {
    cudaError_t e = set_smem_attr<E, QT, GM>(sm);
    if (e != cudaSuccess) return e;
    k_forward_res<E, QT, GM><<<g, b, sm, s>>>(p, it, tape);
    return cudaGetLastError();
  }
  static cudaError_t bwd(dim3 g, dim3 b, size_t sm, cudaStream_t s, const ProbDev* p, const WorkItem* it) {
    cudaError_t e = set_smem_attr<E, QT, GM>(sm);
    if (e != cudaSuccess) return e;
    k_backward_res<E, QT, GM><<<g, b, sm, s>>>(p, it);
    return cudaGetLastError();
  }
  static cudaError_t prop(dim3 g, dim3 b, size_t sm, cudaStream_t s, const ProbDev* p, int adj, int j0, int j1,
                          double2* x) {
    cudaError_t e = set_smem_attr<E, QT, GM>(sm);
    if (e != cudaSuccess) return e;
    k_propagate_res<E, QT, GM><<<g, b, sm, s>>>(p, adj, j0, j1, x);
    return cudaGetLastError();
  }
};

#define LB_RES_DISPATCH(rc, CALL)                       \
  do {                                                  \
    if ((rc).gmres) {                                   \
      switch ((rc).E) {                                 \
        case 1: return ResKernels<1, 0, true>::CALL;    \
        case 2: return ResKernels<2, 0, true>::CALL;    \
        case 4: return ResKernels<4, 0, true>::CALL;    \
        case 8: return ResKernels<8, 0, true>::CALL;    \
        default: return cudaErrorInvalidValue;          \
      }                                                 \
    }                                                   \
    if ((rc).E == 1) {                                  \
      switch ((rc).QT) {                                \
        case 1: return ResKernels<1, 1>::CALL;          \
        case 2: return ResKernels<1, 2>::CALL;          \
        case 3: return ResKernels<1, 3>::CALL;          \
        case 4: return ResKernels<1, 4>::CALL;          \
        default: return ResKernels<1, 0>::CALL;         \
      }                                                 \
    }                                                   \
    switch ((rc).E) {                                   \
      case 2: return ResKernels<2, 0>::CALL;            \
      case 4: return ResKernels<4, 0>::CALL;            \
      case 8: return ResKernels<8, 0>::CALL;            \
      default: return cudaErrorInvalidValue;            \
    }                                                   \
  } while (0)

cudaError_t launch_forward_resident(const ProbDev* d_probs, const WorkItem* d_items, int n_items, int tape,
                                    const ResidentConfig& rc, cudaStream_t s) {
  LB_RES_DISPATCH(rc, fwd(dim3(n_items), dim3(rc.threads), rc.smem, s, d_probs, d_items, tape));
}

cudaError_t launch_backward_resident(const ProbDev* d_probs, const WorkItem* d_items, int n_items,
                                     const ResidentConfig& rc, cudaStream_t s) {
  LB_RES_DISPATCH(rc, bwd(dim3(n_items), dim3(rc.threads), rc.smem, s, d_probs, d_items));
}

cudaError_t launch_propagate_resident(const ProbDev* d_prob, int adjoint, int64_t j0, int64_t j1, double2* x,
                                      int n_vec, const ResidentConfig& rc, cudaStream_t s) {
  LB_RES_DISPATCH(rc, prop(dim3(n_vec), dim3(rc.threads), rc.smem, s, d_prob, adjoint, (int)j0, (int)j1, x));
}

cudaError_t launch_tables(ProbDev* d_prob, const ProbDev& h, cudaStream_t s) {
  int n = h.V > h.njcoef ? h.V : h.njcoef;
  if (h.ncoef > n) n = h.ncoef;
  if (h.N > n) n = h.N;
  k_tables<<<(n + 255) / 256, 256, 0, s>>>(d_prob);
  return cudaGetLastError();
}

cudaError_t launch_gate_targets(const ProbDev& h, const double2* Vg, const int32_t* emap, const int32_t* efull,
                                int32_t Ne, cudaStream_t s) {
  const size_t n = (size_t)h.M * h.V;
  k_gate_targets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h, Vg, emap, efull, Ne);
  return cudaGetLastError();
}

cudaError_t launch_control_table(const ProbDev* d_prob, const ProbDev& h, cudaStream_t s) {
  const size_t n = (size_t)h.NT * h.cq;
  k_control_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_prob);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stop_factors<<<(unsigned)((h.NT + 255) / 256), 256, 0, s>>>(d_prob);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const ProbDev* d_probs, int n_probs, int max_param_warps, int with_grad, cudaStream_t s) {
  k_objective<<<n_probs, 32, 0, s>>>(d_probs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !with_grad) return e;
  k_gproj_reduce<<<dim3(304, n_probs), 256, 0, s>>>(d_probs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int threads = 128;
  dim3 grid((max_param_warps * 32 + threads - 1) / threads, n_probs);
  k_gradient_project<<<grid, threads, 0, s>>>(d_probs);
  return cudaGetLastError();
}

cudaError_t launch_gather(const ProbDev* d_probs, int n_probs, const int64_t* grad_off, double* G_all,
                          double* grad_all, DevStatus* st_all, cudaStream_t s) {
  k_gather<<<n_probs, 128, 0, s>>>(d_probs, grad_off, G_all, grad_all, st_all);
  return cudaGetLastError();
}

cudaError_t launch_apply(const ProbDev* d_prob, const ProbDev& h, int adjoint, int64_t step, const double2* x,
                         double2* y, int n_vec, cudaStream_t s) {
  const size_t n = (size_t)n_vec * h.V;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (adjoint)
    k_apply<true><<<blocks, 256, 0, s>>>(d_prob, (int)step, x, y, n_vec);
  else
    k_apply<false><<<blocks, 256, 0, s>>>(d_prob, (int)step, x, y, n_vec);
  return cudaGetLastError();
}

size_t grid_smem_bytes(int ncoef, int njcoef) { return grid_smem_bytes_impl(ncoef, njcoef); }

int grid_blocks_max(size_t smem) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_sweep_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k_backward_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int a = 0, b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_sweep_grid, kGridThreads, smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_backward_grid, kGridThreads, smem) != cudaSuccess) return 0;
  per = a < b ? a : b;
  int n = nsm * per;
  return n < kMaxGridBlocks ? n : kMaxGridBlocks;
}

cudaError_t launch_sweep_grid(const ProbDev* d_prob, int mode, int init_from_q0, int tape, int64_t j0, int64_t j1,
                              double2* x, int nstates, int nblocks, size_t smem, cudaStream_t s) {
  int m = mode, in = init_from_q0, tp = tape, a = (int)j0, b = (int)j1, ns = nstates;
  const ProbDev* p = d_prob;
  double2* xx = x;
  void* args[] = {(void*)&p, (void*)&m, (void*)&in, (void*)&tp, (void*)&a, (void*)&b, (void*)&xx, (void*)&ns};
  return cudaLaunchCooperativeKernel((const void*)k_sweep_grid, dim3(nblocks), dim3(kGridThreads), args, smem, s);
}

cudaError_t launch_backward_grid(const ProbDev* d_prob, int nblocks, size_t smem, cudaStream_t s) {
  const ProbDev* p = d_prob;
  void* args[] = {(void*)&p};
  return cudaLaunchCooperativeKernel((const void*)k_backward_grid, dim3(nblocks), dim3(kGridThreads), args, smem, s);
}

cudaError_t launch_objective_states(const ProbDev* d_prob, int M, cudaStream_t s) {
  k_objective_states<<<M, 256, 0, s>>>(d_prob);
  return cudaGetLastError();
}

// ---- cluster-split sweeps ----------------------------------------------------

ClusterConfig cluster_config(int V, int Q, int ncoef, int njcoef, int N, bool cs) {
  ClusterConfig cc{};
  if (Q < 1 || Q > 4) return cc;
  const int L = cs ? (4 * Q <= 4 ? 4 : (4 * Q <= 8 ? 8 : 16)) : (2 * Q <= 2 ? 2 : (2 * Q <= 4 ? 4 : 8));
  const int C = (V * L + 127) / 128;
  if (C < 1 || C > 8) return cc;
  const int Vc = (V + C - 1) / C;
  cc.C = C;
  cc.QT = Q;
  cc.cs = cs;
  cc.threads = ((Vc * L + 31) / 32) * 32;
  cc.smem = cl_smem_bytes(ncoef, njcoef, N, V);
  return cc;
}

template <int QT, bool CS>
struct ClKernels {
  template <class K, class... Args>
  static cudaError_t launch(K kern, const ClusterConfig& cc, int n_states, cudaStream_t s, Args... args) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cc.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_states * cc.C);
    cfg.blockDim = dim3(cc.threads);
    cfg.dynamicSmemBytes = cc.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cc.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
  }
};

#define LB_CL_DISPATCH_CS(cc, CS_, ...)                                          \
  switch ((cc).QT) {                                                             \
    case 1: { constexpr int QT_ = 1; constexpr bool CSV_ = CS_; __VA_ARGS__ }    \
    case 2: { constexpr int QT_ = 2; constexpr bool CSV_ = CS_; __VA_ARGS__ }    \
    case 3: { constexpr int QT_ = 3; constexpr bool CSV_ = CS_; __VA_ARGS__ }    \
    case 4: { constexpr int QT_ = 4; constexpr bool CSV_ = CS_; __VA_ARGS__ }    \
    default: return cudaErrorInvalidValue;                                       \
  }
#define LB_CL_DISPATCH(cc, ...)                 \
  do {                                          \
    if ((cc).cs) {                              \
      LB_CL_DISPATCH_CS(cc, true, __VA_ARGS__)  \
    } else {                                    \
      LB_CL_DISPATCH_CS(cc, false, __VA_ARGS__) \
    }                                           \
  } while (0)

cudaError_t launch_forward_cluster(const ProbDev* d_prob, int M, int tape, const ClusterConfig& cc, cudaStream_t s) {
  LB_CL_DISPATCH(cc, return cc.pen ? ClKernels<QT_, CSV_>::launch(k_forward_cl<QT_, CSV_, true>, cc, M, s, d_prob, tape)
                                   : ClKernels<QT_, CSV_>::launch(k_forward_cl<QT_, CSV_, false>, cc, M, s, d_prob,
                                                                  tape););
}

cudaError_t launch_backward_cluster(const ProbDev* d_prob, int M, const ClusterConfig& cc, cudaStream_t s) {
  LB_CL_DISPATCH(cc, return cc.pen ? ClKernels<QT_, CSV_>::launch(k_backward_cl<QT_, CSV_, true>, cc, M, s, d_prob)
                                   : ClKernels<QT_, CSV_>::launch(k_backward_cl<QT_, CSV_, false>, cc, M, s, d_prob););
}

cudaError_t launch_propagate_cluster(const ProbDev* d_prob, int adjoint, int64_t j0, int64_t j1, double2* x, int n_vec,
                                     const ClusterConfig& cc, cudaStream_t s) {
  LB_CL_DISPATCH(cc, return ClKernels<QT_, CSV_>::launch(k_propagate_cl<QT_, CSV_>, cc, n_vec, s, d_prob, adjoint,
                                                        (int)j0, (int)j1, x););
}

}  // namespace lbk
