// One-CTA-per-state sweeps (the state in shared memory, the whole time loop
// in one launch), their GMRES inner solve and their launchers.

#include "lb_device.cuh"

namespace lbk {

namespace {

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
      const uint32_t t = P.hkl[i];
      const int k = (int)(t & 0xffffu), l = (int)(t >> 16), v = k + P.N * l;
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
// cl receives, per element, the correction (dt/2) O z of the last iteration's
// input (the correction whose Jacobi image is the returned z; not written by
// GMRES), which the predictor records.
template <int E, int QT, bool ADJ, bool GM = false>
__device__ int res_solve(const ResSmem& S, const Hdr& H, const Elems<E>& el, const Plan<QT>& pl,
                         const double2 (&rhs)[E], const double2* __restrict__ ct, double fac, int& cur,
                         double2 (&cl)[E], const double2* pc = nullptr) {
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
        double cr = 0.0, ci = 0.0;
        double2 d;
        if constexpr (QT > 0) {
          offdiag_plan<QT, ADJ>(cr, ci, zc, pl, cq, jon);
          d = pl.d;
        } else {
          offdiag_acc<ADJ>(cr, ci, zc, v, el.kd[e], el.ld[e], H, T, ct);
          d = S.dsm[v];
        }
        cl[e] = make_double2(cr, ci);
        const double ar = rhs[e].x + cr, ai = rhs[e].y + ci;
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
// previous steps live in the anchored ring P.hist ([kRingOrder][M * V], this
// state's elements at base + v) with the powers g^m, g^-m of its frame
// (P.hgp, P.hgm) and are extrapolated in each element's rotating frame
// (anchored_sum); every element is read and written by the thread that owns
// it, so no synchronisation is needed.
template <int E>
struct Pred {
  double2* hist = nullptr;
  double2* gp = nullptr;  // g^m per element of this state
  double2* gm = nullptr;  // g^-m
  const double2* D = nullptr;
  const double2* Ginv = nullptr;
  size_t stride = 0;
  double hh = 0.0;
  int n = 0, slot = 0, cap = kRingOrder;  // cap: the predictor's order
  int m = 0;                              // steps since the anchor
  __device__ void init(const ProbDev& P, size_t base) {
    use(P.hist + base, P.hgp + base, P.hgm + base);
    D = P.D;
    Ginv = P.Ginv;
    stride = (size_t)P.M * P.V;
    hh = 0.5 * P.h;
    n = slot = m = 0;
    cap = P.pred_order;
  }
  __device__ void use(double2* ring, double2* p, double2* q) {
    hist = ring;
    gp = p;
    gm = q;
  }
  __device__ void restart() {
    n = 0;
    m = 0;
  }
  // pc[e]: the predicted correction of element e; a fresh anchor (n = 0)
  // resets the element's powers
  __device__ void predict(double2 (&pc)[E], const Elems<E>& el, const ResSmem& S, const Hdr& H, int V) const {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      pc[e] = make_double2(0.0, 0.0);
      if (v < V) {
        if (n > 0) {
          pc[e] = cmul(gp[v], anchored_sum(hist + v, stride, slot, n));
        } else {
          gp[v] = make_double2(1.0, 0.0);
          gm[v] = make_double2(1.0, 0.0);
        }
      }
    }
  }
  // the end of a step: its corrections c into the anchor frame, the powers
  // advanced by g (S.dsm holds (I - dt/2 D)^-1, so g = 2 S.dsm - 1; ADJ: the
  // conjugate factor), and every kAnchorSteps steps the anchor moved to the
  // next step
  template <bool ADJ>
  __device__ void commit(const double2 (&c)[E], const Elems<E>& el, const ResSmem& S, const Hdr& H, int V) {
    const bool re = m + 1 >= kAnchorSteps;
    const int nn = n < cap ? n + 1 : cap;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      if (v < V) {
        const double2 gpv = gp[v], gmv = gm[v];
        hist[(size_t)slot * stride + v] = cmul(c[e], gmv);
        const double2 d = S.dsm[v], gi = __ldg(Ginv + v);
        const double2 g = make_double2(fma(2.0, d.x, -1.0), ADJ ? -2.0 * d.y : 2.0 * d.y);
        double2 np = cmul(gpv, g), nm = cmul(gmv, make_double2(gi.x, ADJ ? -gi.y : gi.y));
        if (re) {
          // the next step becomes the anchor: the ring's entries times g^(m+1)
          int sl = slot;
          for (int i = 0; i < nn; ++i) {
            double2* r = hist + (size_t)sl * stride + v;
            *r = cmul(*r, np);
            sl = sl > 0 ? sl - 1 : kRingOrder - 1;
          }
          np = make_double2(1.0, 0.0);
          nm = np;
        }
        gp[v] = np;
        gm[v] = nm;
      }
    }
    n = nn;
    slot = slot + 1 < kRingOrder ? slot + 1 : 0;
    m = re ? 0 : m + 1;
  }
  // record the corrections the last inner iteration computed (fixed points)
  template <bool ADJ>
  __device__ void record_c(const double2 (&cl)[E], const Elems<E>& el, const ResSmem& S, const Hdr& H, int V) {
    commit<ADJ>(cl, el, S, H, V);
  }
  // record c = (I - dt/2 D) z - rhs from the solution (GMRES)
  template <bool ADJ>
  __device__ void record(const double2* zc, const double2 (&rhs)[E], const Elems<E>& el, const ResSmem& S,
                         const Hdr& H, int V) {
    double2 c[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      c[e] = make_double2(0.0, 0.0);
      if (v < V) {
        const double2 z = zc[v], d = __ldg(D + v);
        const double dr = hh * d.x, di = hh * (ADJ ? -d.y : d.y);
        c[e] = make_double2(z.x - fma(dr, z.x, -di * z.y) - rhs[e].x, z.y - fma(dr, z.y, di * z.x) - rhs[e].y);
      }
    }
    commit<ADJ>(c, el, S, H, V);
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
  // With the Hermitian symmetry every Krylov vector is Hermitian (the
  // preconditioned operator maps Hermitian matrices to Hermitian ones), so the
  // inner products over all N^2 entries are real: the k <= l entries are
  // summed with weight 2 off the diagonal and the imaginary parts vanish;
  // vectors are written at (k, l) and, conjugated, at the mirror (l, k).
  const bool hm = H.herm != 0;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  double* gm = S.gm;
  double2* kry = S.kry;
  const double2* rhs = S.zb1;
  double2* xs = S.zb0;
  double2 x[E];
  // weight of element e in the inner products
  auto wt = [&](int e) { return el_m(el, S, H, e) >= 0 ? 2.0 : 1.0; };
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int v = el_v(el, S, H, e);
    x[e] = v < V ? xs[v] : make_double2(0.0, 0.0);
  }
  int its = 0;
  for (;;) {
    // r = Dinv (q + dt/2 O z) - z, normalised into the first basis vector
    double nrm = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int v = el_v(el, S, H, e);
      if (v < V) {
        double ar = rhs[v].x, ai = rhs[v].y;
        offdiag_acc<ADJ>(ar, ai, xs, v, el.kd[e], el.ld[e], H, T, ct);
        const double2 d = S.dsm[v];
        const double di = ADJ ? -d.y : d.y;
        const double2 r = make_double2(fma(d.x, ar, -di * ai) - x[e].x, fma(d.x, ai, di * ar) - x[e].y);
        rputm(kry, v, el_m(el, S, H, e), r);
        nrm = fma(wt(e), fma(r.x, r.x, r.y * r.y), nrm);
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
      const int v = el_v(el, S, H, e);
      if (v < V) rputm(kry, v, el_m(el, S, H, e), make_double2(kry[v].x * ib, kry[v].y * ib));
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
        const int v = el_v(el, S, H, e);
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
            const int v = el_v(el, S, H, e);
            if (v < V) {
              const double2 u = kry[(size_t)i * V + v];
              if (hm) {
                sr = fma(wt(e), fma(u.x, w[e].x, u.y * w[e].y), sr);
              } else {
                sr = fma(u.x, w[e].x, fma(u.y, w[e].y, sr));
                si = fma(u.x, w[e].y, fma(-u.y, w[e].x, si));
              }
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
            const int v = el_v(el, S, H, e);
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
      for (int e = 0; e < E; ++e) n2 = fma(wt(e), fma(w[e].x, w[e].x, w[e].y * w[e].y), n2);
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
        const int v = el_v(el, S, H, e);
        if (v < V) rputm(vn, v, el_m(el, S, H, e), make_double2(w[e].x * ih, w[e].y * ih));
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
      const int v = el_v(el, S, H, e);
      if (v < V) {
        double2 z = x[e];
        for (int i = 0; i < k; ++i) {
          const double yr = gm[kGmY + 2 * i], yi = gm[kGmY + 2 * i + 1];
          const double2 u = kry[(size_t)i * V + v];
          z.x += fma(yr, u.x, -yi * u.y);
          z.y += fma(yr, u.y, yi * u.x);
        }
        x[e] = z;
        rputm(xs, v, el_m(el, S, H, e), z);
      }
    }
    __syncthreads();
    if (conv) return its;
    if (its >= H.max_iter) return -1;
  }
}

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
  // first-iterate predictor, forgetting its history at every step j with
  // j % R == 0 (R > 0 divides K, so every checkpoint is a restart point and a
  // recompute repeats these iterates bit for bit)
  const int R = P.pred_restart;
  const bool pred = R >= 0;
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
    if (pred) {
      if (R > 0 && j % R == 0) pr.restart();
      pr.predict(pc, el, S, H, V);
    }
    // pc: the prediction in, the last iteration's corrections out
    const int it = res_solve<E, QT, false, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur, pc,
                                                 pred ? pc : nullptr);
    if (it < 0) {
      if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
      stats.flush(P.status);
      return;
    }
    stats.add(0, it);
    const double2* zc = cur ? S.zb1 : S.zb0;
    if (pred) {
      if (H.method == LB_SOLVER_GMRES)
        pr.template record<false>(zc, q, el, S, H, V);
      else
        pr.template record_c<false>(pc, el, S, H, V);
    }
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
  // the forward predictor of the recompute, restarted as in the forward sweep
  // (at every checkpoint, and at every step j with j % R == 0); it has its own
  // history ring, and the adjoint's ring position is kept across it
  const int R = P.pred_restart;
  const bool fpred = H.K > 0 && R > 0;
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
      const int an = pr.n, aslot = pr.slot, am = pr.m;
      if (fpred) {
        pr.use(P.histf + base, P.fgp + base, P.fgm + base);
        pr.slot = 0;
      }
      for (int j = j0; j < j1; ++j) {
        int cur;
        if (fpred) {
          if (j % R == 0) pr.restart();
          pr.predict(pc, el, S, H, V);
        }
        const int it = res_solve<E, QT, false, GM>(S, H, el, pl, qf, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur,
                                                   pc, fpred ? pc : nullptr);
        if (it < 0) {
          if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
          stats.flush(P.status);
          return;
        }
        stats.add(1, it);
        const double2* zc = cur ? S.zb1 : S.zb0;
        if (fpred) {
          if (H.method == LB_SOLVER_GMRES)
            pr.template record<false>(zc, qf, el, S, H, V);
          else
            pr.template record_c<false>(pc, el, S, H, V);
        }
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
      if (fpred) {
        pr.use(P.hist + base, P.hgp + base, P.hgm + base);
        pr.n = an;
        pr.slot = aslot;
        pr.m = am;
      }
    }
    for (int j = j1 - 1; j >= j0; --j) {
      const double2* ct = P.ctab + (size_t)j * H.cq;
      int cur;
      // (I - dt/2 (M^{j+1/2})^+) zhat^j = qhat^{j+1}   (eq. linsystem_adjoint)
      if (apred) pr.predict(pc, el, S, H, V);
      const int it = res_solve<E, QT, true, GM>(S, H, el, pl, lam, ct, stop_factor(P, j), cur, pc, apred ? pc : nullptr);
      if (it < 0) {
        if (threadIdx.x == 0) record_error(P.status, it == -1 ? LB_ENOTCONV : LB_ENAN, j);
        stats.flush(P.status);
        return;
      }
      stats.add(2, it);
      const double2* zh = cur ? S.zb1 : S.zb0;
      if (apred) {
        if (H.method == LB_SOLVER_GMRES)
          pr.template record<true>(zh, lam, el, S, H, V);
        else
          pr.template record_c<true>(pc, el, S, H, V);
      }
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
            // A = Z conj(R) to g_a and B = Z conj(P) to g_ad
            if (!H.herm) {
              sar = fma(Z[e].x, rr, fma(Z[e].y, ri, sar));
              sai = fma(Z[e].y, rr, fma(-Z[e].x, ri, sai));
              sdr = fma(Z[e].x, pr, fma(Z[e].y, pi, sdr));
              sdi = fma(Z[e].y, pr, fma(-Z[e].x, pi, sdi));
            } else if (el_m(el, S, H, e) >= 0) {
              // Hermitian Z and zhat: the element and its mirror (l, k) add
              // A - conj(B) to the g_a sum and B - conj(A), its negated
              // conjugate, to the g_ad sum
              const double dr = rr - pr, di = ri - pi, ur = rr + pr, ui = ri + pi;
              sar = fma(Z[e].x, dr, fma(Z[e].y, di, sar));
              sai = fma(Z[e].y, ur, fma(-Z[e].x, ui, sai));
            } else {
              // a diagonal element of Hermitian Z and zhat has conj(R) = -P, so
              // B = -conj(A): it adds A to g_a and its negated conjugate to g_ad
              sar = fma(Z[e].x, rr, fma(Z[e].y, ri, sar));
              sai = fma(Z[e].y, rr, fma(-Z[e].x, ri, sai));
            }
          }
        }
        if (H.herm) {
          // the g_ad sum of Hermitian Z and zhat is minus the conjugate of the g_a sum
          sdr = -sar;
          sdi = sai;
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
    double2 cl[E];
    const int it = adjoint ? res_solve<E, QT, true, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur, cl)
                           : res_solve<E, QT, false, GM>(S, H, el, pl, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), cur, cl);
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

}  // namespace lbk
