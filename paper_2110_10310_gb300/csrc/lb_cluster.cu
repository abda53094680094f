// Cluster-split sweeps for small states (one thread-block cluster per state)
// and their launchers.

#include "lb_device.cuh"

namespace lbk {

namespace {

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
  int vm;       // under the Hermitian symmetry the element's mirror l + N k (k < l), else -1
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

// herm: the Hermitian symmetry -- the cluster's lanes take the elements
// k <= l only (column by column), each pushing its value to its mirror too
template <int QT, bool CS>
__device__ ClPlan cl_plan(const ClSmem& S, int C, int crank, bool herm) {
  constexpr int L = ClLanes<QT, CS>::L;
  const Hdr& H = *S.hdr;
  const int Ve = herm ? H.N * (H.N + 1) / 2 : H.V;  // elements the sweep computes
  const int Vc = (Ve + C - 1) / C;
  const int le = threadIdx.x / L;
  ClPlan pl;
  pl.r = threadIdx.x % L;
  const int idx = crank * Vc + le;
  pl.ev = le < Vc && idx < Ve;
  int v = idx, vm = -1;
  if (herm && pl.ev) {
    // packed index idx = l (l + 1) / 2 + k, k <= l
    int l = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
    while ((l + 1) * (l + 2) / 2 <= idx) ++l;
    while (l * (l + 1) / 2 > idx) --l;
    const int k = idx - l * (l + 1) / 2;
    v = k + H.N * l;
    vm = k != l ? l + H.N * k : -1;
  }
  pl.v = pl.ev ? v : 0;
  pl.vm = pl.ev ? vm : -1;
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
  unsigned zbm[2], zsm[2];  // the element's mirror (Hermitian symmetry)
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
    const int vm = pl.vm >= 0 ? pl.vm : pl.v;
    A.zbm[b] = mapa_u32(smem_u32(S.zb + (size_t)b * V + vm), rr0);
    A.zsm[b] = mapa_u32(smem_u32(S.zs + (size_t)b * V + vm), rr0);
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
    // under the Hermitian symmetry the element's mirror gets the conjugate,
    // so every entry of the replicas is still written once per exchange
    const bool mir = pl.vm >= 0;
    st_async_f64x2(A.zb[p], z.x, z.y, A.mb[p]);
    if (mir) st_async_f64x2(A.zbm[p], z.x, -z.y, A.mb[p]);
    if (spec) {
      st_async_f64x2(A.zs[sb], zn.x, zn.y, A.mb[p]);
      if (mir) st_async_f64x2(A.zsm[sb], zn.x, -zn.y, A.mb[p]);
    }
    const unsigned dst = smem_u32(S.zb + (size_t)p * V + pl.v);
    const unsigned dsp = smem_u32(S.zs + (size_t)sb * V + pl.v);
    const unsigned dstm = smem_u32(S.zb + (size_t)p * V + (mir ? pl.vm : pl.v));
    const unsigned dspm = smem_u32(S.zs + (size_t)sb * V + (mir ? pl.vm : pl.v));
    for (int cc = pl.r + L; cc < C; cc += L) {
      const unsigned mbr = mapa_u32(mb_local, cc);
      st_async_f64x2(mapa_u32(dst, cc), z.x, z.y, mbr);
      if (mir) st_async_f64x2(mapa_u32(dstm, cc), z.x, -z.y, mbr);
      if (spec) {
        st_async_f64x2(mapa_u32(dsp, cc), zn.x, zn.y, mbr);
        if (mir) st_async_f64x2(mapa_u32(dspm, cc), zn.x, -zn.y, mbr);
      }
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
    // an off-diagonal element under the symmetry stands for its mirror too
    if (pl.vm >= 0) P.qT[base + pl.vm] = make_double2(q.x, -q.y);
    const double2 t = P.tar[base + pl.v];
    if (H.kind == LB_J_FROB) {
      const double dr = q.x - t.x, dq = q.y - t.y;
      acc = fma(dr, dr, dq * dq);
    } else {
      acc = fma(t.x, q.x, t.y * q.y);
    }
    if (pl.vm >= 0) acc *= 2.0;
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
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank, H.herm != 0);
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
  // the predictor is used only when no step is ever recomputed (K == 0: the
  // recompute of this sweep starts every solve cold, and recomputed stage
  // vectors must stay bit-identical to the forward ones), restarted at every
  // step j with j % R == 0 for R > 0
  const int R = P.pred_restart;
  const bool pred = H.K == 0 && R >= 0;
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
      if (own) pacc = fma(st.pen * (pl.vm >= 0 ? 2.0 : 1.0), cl_merit_summand(H.kind, rhs, tv), pacc);
      ppen += st.pen;
    }
    ClHist hn = hist;
    if (hist.on) {
      hn.advance();
      if (R > 0 && (j + 1) % R == 0) hn.n = 0;
    }
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
  const bool herm = H.herm != 0;
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank, herm);
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
      if (herm) {
        // Hermitian Z and zhat: an off-diagonal element and its mirror add
        // A - conj(B) to g_a and B - conj(A) to g_ad (A = Z conj(R) on the
        // R half's lanes, B = Z conj(P) on the P half's), i.e. each half's
        // value minus the conjugate of the other half's; a diagonal element
        // has B = -conj(A) already.  The other half of the same subsystem
        // (and component) is lane r ^ 1, or r ^ 2 with the component split.
        constexpr int pm = CS ? 2 : 1;
        const double osr = __shfl_xor_sync(kFull, sr, pm), osi = __shfl_xor_sync(kFull, si, pm);
        if (gl && pl.vm >= 0 && pl.q < Qn) {
          if constexpr (CS) {
            sr = (pl.r & 1) ? sr + osr : sr - osr;
          } else {
            sr -= osr;
            si += osi;
          }
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
  const ClPlan pl = cl_plan<QT, CS>(S, C, crank, false);  // vectors given to lb_propagate may be anything
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

}  // namespace

// ---------------------------------------------------------------------------
// launchers

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
