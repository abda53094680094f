// Grid-wide cooperative sweeps for states too large for one CTA, and their
// launchers.

#include "lb_device.cuh"

namespace lbk {

namespace {

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

// Neighbour reads of the iterates go through L1 (kNbL2 = false): each value
// is read by up to 1 + 5Q elements, most of them in the same block's chunk.
// The iterates are rewritten by other blocks between iterations; every such
// read follows a grid_sync, whose fence after the wait (acquire, GPU scope)
// makes the writes of the previous iteration visible to ordinary loads (the
// ordering cooperative groups' grid sync provides with the same pattern).
constexpr bool kNbL2 = false;

// Grid barrier with a bounded wait: at most `limit` polls (kSpinLimit unless
// the handle set another bound, lb_set_wait_limit).  Returns false on every
// block once a wait has given up (the kernel then returns).
__device__ bool grid_sync(GridBar* bar, unsigned nblocks, long long limit) {
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
        if (++spins > limit) {
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
  int herm;         // Hermitian symmetry: only elements k <= l are iterated and stored
  int Vh;           // elements per state in the loops and in the sweep's own buffers: V, or N (N + 1) / 2
  long long total;  // M * Vh
  long long chunk;  // elements per block
};

// Element e of a grid sweep's loops: state b, vec index v = k + N l, and i,
// its place in the state's slab of the sweep's own buffers (iterates,
// adjoint, recomputed state, checkpoints, segment tape, predictor rings).
// Without the symmetry the slab is the vec layout (i = v).  With it the loops
// visit k <= l only ((k, l) from the table hkl) and the slabs hold those entries
// packed, column by column (i = l (l + 1)/2 + k); vm is then the mirror index
// l + N k of an off-diagonal element in the vec layout of the inputs and
// outputs (q0, targets, final states), whose value is the conjugate (-1 for
// diagonal elements and without the symmetry).
struct GEl {
  int b, v, vm, i, k, l;
};
// element i of state b's slab
__device__ __forceinline__ GEl gel_at(const GridHdr& G, const uint32_t* __restrict__ hkl, int b, int i) {
  GEl r;
  const int N = G.h.N;
  r.b = b;
  r.i = i;
  if (!G.herm) {
    r.v = i;
    r.vm = -1;
    r.k = i % N;
    r.l = i / N;
    return r;
  }
  const uint32_t t = __ldg(hkl + i);
  r.k = (int)(t & 0xffffu);
  r.l = (int)(t >> 16);
  r.v = r.k + N * r.l;
  r.vm = r.k != r.l ? r.l + N * r.k : -1;
  return r;
}

// A thread's walk over its elements e = e0 + threadIdx.x, + blockDim.x, ...
// of a block's chunk [e0, e1) of the flattened [M][Vh] range, keeping the
// state b and slab index i of e (one division at the start).
struct GIter {
  long long e;
  int b, i;
  __device__ GIter(const GridHdr& G, long long e_start) : e(e_start) {
    b = (int)(e / G.Vh);
    i = (int)(e - (long long)b * G.Vh);
  }
  __device__ __forceinline__ void next(const GridHdr& G, int step) {
    e += step;
    i += step;
    while (i >= G.Vh) {
      i -= G.Vh;
      ++b;
    }
  }
};

// offset of element g in slab `slab` (state b's, or a checkpoint's) of a sweep buffer
__device__ __forceinline__ size_t gslab(const GridHdr& G, const GEl& g, size_t slab) {
  return slab * (size_t)G.Vh + g.i;
}
// store x at element g of an input/output array in the vec layout (and its mirror)
__device__ __forceinline__ void gput(double2* a, const GEl& g, int V, double2 x) {
  a[(size_t)g.b * V + g.v] = x;
  if (g.vm >= 0) a[(size_t)g.b * V + g.vm] = make_double2(x.x, -x.y);
}

// entries of one step of the control table at most: Q factors and the pairs p < q
constexpr int kMaxCq = LB_MAXQ + LB_MAXQ * (LB_MAXQ - 1) / 2;

// z as a pair of single-precision numbers (hi, lo) with hi + lo = z to about
// 2^-48 |z| (lb_set_precision): hi is z truncated to 24 significant bits, lo
// the remaining 29 bits rounded to 24.  |z| below 2^-126 is flushed to zero,
// and lo is dropped for |z| below 2^-74 (an absolute error under 2^-98).
// Integer pipe except one conversion and one multiplication by a power of
// two.
__device__ __forceinline__ float2 split_f64(double z) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(z);
  const unsigned sgn = (unsigned)(bits >> 32) & 0x80000000u;
  const int E = (int)((bits >> 52) & 0x7ff);
  const int eh = E - 896;  // single-precision exponent field of hi
  const float hi = __uint_as_float(eh <= 0 ? sgn : (sgn | ((unsigned)min(eh, 254) << 23) |
                                                    ((unsigned)(bits >> 29) & 0x7fffffu)));
  const int el = E - 948;  // exponent field of 2^(E - 1075), the weight of the mantissa's last bit
  const float lo = (eh <= 0 || el <= 0) ? 0.0f
                                        : __uint2float_rn((unsigned)bits & 0x1fffffffu) *
                                              __uint_as_float((unsigned)min(el, 254) << 23);
  return make_float2(hi, sgn ? -lo : lo);
}

__host__ __device__ inline size_t grid_smem_bytes_impl(int ncoef, int njcoef) {
  return align16(sizeof(GridHdr)) + align16(sizeof(double) * 2 * ncoef) + align16(sizeof(double) * 2 * njcoef) +
         align16(sizeof(float) * 2 * ncoef) + align16(sizeof(float) * 2 * njcoef) + align16(sizeof(float2) * kMaxCq) +
         align16(sizeof(float2) * 2 * ncoef) + align16(sizeof(float2) * 2 * njcoef) + align16(sizeof(float4) * LB_MAXQ) +
         align16(sizeof(double) * 4 * 8) + 64;
}

struct GridSmem {
  GridHdr* g;
  double* cu;
  double* cd;
  double* jf;
  double* ja;
  float* cuf;  // the same four tables in single precision (difference iterations)
  float* cdf;
  float* jff;
  float* jaf;
  float2* ctf;  // this solve's control-table entries in single precision
  // paired-single tables (lb_set_precision): the ladder factors cu, cd and
  // the decay factors jf, ja as (hi, lo) pairs, and per subsystem this
  // solve's control factor (dt/2) d_q = a + i b as (b hi, b lo, a hi, a lo)
  // (negated for the adjoint)
  float2* ffcu;
  float2* ffcd;
  float2* ffjf;
  float2* ffja;
  float4* ffab;
  double* red;  // [4][8 warps]
  int* flag;    // [0]: the iteration's decision, [1]: next iteration in single precision
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
  S.cuf = reinterpret_cast<float*>(base + o);
  S.cdf = S.cuf + P.ncoef;
  o += align16(sizeof(float) * 2 * P.ncoef);
  S.jff = reinterpret_cast<float*>(base + o);
  S.jaf = S.jff + P.njcoef;
  o += align16(sizeof(float) * 2 * P.njcoef);
  S.ctf = reinterpret_cast<float2*>(base + o);
  o += align16(sizeof(float2) * kMaxCq);
  S.ffcu = reinterpret_cast<float2*>(base + o);
  S.ffcd = S.ffcu + P.ncoef;
  o += align16(sizeof(float2) * 2 * P.ncoef);
  S.ffjf = reinterpret_cast<float2*>(base + o);
  S.ffja = S.ffjf + P.njcoef;
  o += align16(sizeof(float2) * 2 * P.njcoef);
  S.ffab = reinterpret_cast<float4*>(base + o);
  o += align16(sizeof(float4) * LB_MAXQ);
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
    S.cuf[i] = (float)P.cu[i];
    S.cdf[i] = (float)P.cd[i];
    S.ffcu[i] = split_f64(P.cu[i]);
    S.ffcd[i] = split_f64(P.cd[i]);
  }
  for (int i = threadIdx.x; i < P.njcoef; i += blockDim.x) {
    S.jf[i] = P.jf[i];
    S.ja[i] = P.ja[i];
    S.jff[i] = (float)P.jf[i];
    S.jaf[i] = (float)P.ja[i];
    S.ffjf[i] = split_f64(P.jf[i]);
    S.ffja[i] = split_f64(P.ja[i]);
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
// First-iterate predictor of the grid sweeps (the anchored ring of
// lb_device.cuh): the off-diagonal corrections c = (dt/2) O z of the last n
// steps, kept per element in a ring (P.hist, or P.histf for the forward
// predictor of a recompute; each element always handled by the same thread,
// so no synchronisation is needed), with the powers g^m and g^-m of its
// anchor frame per element (gp, gm).
struct GridHist {
  double2* ring = nullptr;
  double2* gp = nullptr;  // g^m per element (slab layout)
  double2* gm = nullptr;  // g^-m
  int n = 0, slot = 0, cap = kRingOrder;  // cap: the predictor's order
  int m = 0;                              // steps since the anchor
  __device__ void advance() {
    n = n < cap ? n + 1 : cap;
    slot = slot + 1 < kRingOrder ? slot + 1 : 0;
    ++m;
  }
  __device__ void restart() {
    n = 0;
    m = 0;
  }
};

// After a step has converged, for element o (slab offset) at vec index v:
// bring the correction the last iteration recorded into the anchor frame
// and advance the powers of g to the next step (ADJ: the conjugate factor);
// every kAnchorSteps steps move the anchor to the next step.  `h` is the
// ring's state before advance().
template <bool ADJ>
__device__ __forceinline__ void grid_commit(const ProbDev& P, const GridHist& h, size_t o, size_t stride, int v) {
  double2* cs = h.ring + (size_t)h.slot * stride + o;
  const double2 gmv = h.gm[o], gpv = h.gp[o];
  *cs = cmul(*cs, gmv);
  const double2 d = __ldg(P.Dinv + v), gi = __ldg(P.Ginv + v);
  const double2 g = make_double2(fma(2.0, d.x, -1.0), ADJ ? -2.0 * d.y : 2.0 * d.y);
  const double2 ginv = make_double2(gi.x, ADJ ? -gi.y : gi.y);
  double2 gp = cmul(gpv, g), gm = cmul(gmv, ginv);
  if (h.m + 1 >= kAnchorSteps) {
    // the next step becomes the anchor: the ring's entries times g^(m+1)
    const int nn = h.n < h.cap ? h.n + 1 : h.cap;
    int sl = h.slot;
    for (int i = 0; i < nn; ++i) {
      double2* c = h.ring + (size_t)sl * stride + o;
      *c = cmul(*c, gp);
      sl = sl > 0 ? sl - 1 : kRingOrder - 1;
    }
    gp = make_double2(1.0, 0.0);
    gm = gp;
  }
  h.gp[o] = gp;
  h.gm[o] = gm;
}

// Running penalty (Sec. III, eq. optimproblem): with penw != 0 the first
// pass of a forward solve also sums each state's merit summand of its
// right-hand side q^j against the target, per block for the (at most
// kLocalStates) states of the block's chunk; after the first grid barrier
// block 0 adds penw * J(q^j) to P.jpen per state, summing the blocks in a
// fixed order.
__device__ __forceinline__ double merit_summand(int kind, double2 q, double2 t) {
  if (kind == LB_J_FROB) {
    const double dr = q.x - t.x, di = q.y - t.y;
    return fma(dr, dr, di * di);
  }
  return fma(t.x, q.x, t.y * q.y);
}

// ---------------------------------------------------------------------------
// Difference iterations (lb_set_difference_iterations).  Once every state's
// last change d = z_k - z_{k-1} is below kDiffRel of its max|q|, the next
// Jacobi iteration computes the change of the correction, (dt/2) O d, and of
// the iterate, (I - dt/2 D)^-1 (dt/2) O d, in single precision from d
// rounded to single precision, and adds them to the FP64 correction and
// iterate: z_{k+1} = z_k + (I - dt/2 D)^-1 (c(z_k) - c(z_{k-1})) is the
// Jacobi step.  Their rounding errors (2^-24 of terms below kDiffRel max|q|)
// stay under the FP64 rounding of z.  The format conversions run on the
// integer pipe (the FP64 pipe bounds the sweeps): truncation to single
// precision, values below its normal range flushed to zero.
constexpr double kDiffRel = 0x1p-32;    // largest change, relative to max|q|, for a difference iteration
constexpr double kDiffFloor = 0x1p-50;  // smallest max|q| for which they are taken

__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  int e = (int)((b >> 52) & 0x7ff) - 896;  // the single-precision exponent field
  e = e > 254 ? 255 : e;                   // out of range: infinity (not reached where used)
  const unsigned man = e == 255 ? 0u : (unsigned)(b >> 29) & 0x7fffffu;
  return __uint_as_float(e <= 0 ? sgn : (sgn | ((unsigned)e << 23) | man));
}
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long ed = e == 255u ? 2047ull : (unsigned long long)(e + 896u);
  const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(e == 0u ? sgn : (sgn | (ed << 52) | man)));
}
// entry (k, l) of a packed Hermitian difference (as ldpk)
__device__ __forceinline__ float2 ldpkf(const float2* p, int k, int l) {
  const bool lo = k > l;
  const int a = lo ? l : k, c = lo ? k : l;
  const float2* q = p + ((c * (c + 1)) >> 1) + a;
  float2 x = kNbL2 ? __ldcg(q) : *q;
  x.y = __uint_as_float(__float_as_uint(x.y) ^ (lo ? 0x80000000u : 0u));
  return x;
}

// offdiag_acc in single precision on a difference d (the same terms: the
// control commutators, the decay sandwich and the Jaynes-Cummings pairs).
// QN = H.Q as a compile-time count, so that the subsystem loop unrolls and
// every neighbour load can be issued before the arithmetic: with little
// arithmetic per load this pass is bound by the latency of L2 reads.
template <bool ADJ, bool PK, int QN>
__device__ __forceinline__ void offdiag_acc_f(float& ar, float& ai, const float2* __restrict__ x, int v, uint32_t kd,
                                              uint32_t ld, const Hdr& H, const GridSmem& S, int k, int l) {
  const int N = H.N;
  auto nb = [&](int dk, int dl) -> float2 {
    if constexpr (PK) return ldpkf(x, k + dk, l + dl);
    else return kNbL2 ? __ldcg(x + v + dk + dl * N) : x[v + dk + dl * N];
  };
#pragma unroll
  for (int q = 0; q < QN; ++q) {
    const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
    const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
    const float c1 = S.cuf[co + nk], c2 = S.cdf[co + nl], c3 = S.cdf[co + nk], c4 = S.cuf[co + nl];
    const float2 x1 = nb(nk + 1 < n ? s : 0, 0);
    const float2 x2 = nb(0, nl > 0 ? -s : 0);
    const float2 x3 = nb(nk > 0 ? -s : 0, 0);
    const float2 x4 = nb(0, nl + 1 < n ? s : 0);
    const float pr = fmaf(-c2, x2.x, c1 * x1.x);
    const float pi = fmaf(-c2, x2.y, c1 * x1.y);
    const float rr = fmaf(-c4, x4.x, c3 * x3.x);
    const float ri = fmaf(-c4, x4.y, c3 * x3.y);
    const float ur = pr + rr, ui = pi + ri, wr = pr - rr, wi = pi - ri;
    const float2 c = S.ctf[q];
    const float a = ADJ ? -c.x : c.x, b = ADJ ? -c.y : c.y;
    ar = fmaf(b, wr, fmaf(a, ui, ar));
    ai = fmaf(b, wi, fmaf(-a, ur, ai));
    if ((H.jon >> q) & 1u) {
      const int jo = H.joff[q] + nk * n + nl;
      float cj;
      float2 x5;
      if (!ADJ) {
        cj = S.jff[jo];
        const int d = (nk + 1 < n && nl + 1 < n) ? s : 0;
        x5 = nb(d, d);
      } else {
        cj = S.jaf[jo];
        const int d = (nk > 0 && nl > 0) ? s : 0;
        x5 = nb(-d, -d);
      }
      ar = fmaf(cj, x5.x, ar);
      ai = fmaf(cj, x5.y, ai);
    }
  }
  for (int kp = 0; kp < H.npair; ++kp) {
    const int p = H.jp[kp], q = H.jq[kp];
    const int np = H.lev[p], nq = H.lev[q], sp = H.stride[p], sq = H.stride[q];
    const int pk = (kd >> (H.db * p)) & H.dm, qk = (kd >> (H.db * q)) & H.dm;
    const int pl = (ld >> (H.db * p)) & H.dm, ql = (ld >> (H.db * q)) & H.dm;
    const float u1 = S.cdf[H.coff[p] + pk] * S.cuf[H.coff[q] + qk];
    const float u2 = S.cuf[H.coff[p] + pl] * S.cdf[H.coff[q] + ql];
    const float w1 = S.cuf[H.coff[p] + pk] * S.cdf[H.coff[q] + qk];
    const float w2 = S.cdf[H.coff[p] + pl] * S.cuf[H.coff[q] + ql];
    const int d = sq - sp;
    const float2 xu1 = nb((pk > 0 && qk + 1 < nq) ? d : 0, 0);
    const float2 xu2 = nb(0, (ql > 0 && pl + 1 < np) ? -d : 0);
    const float2 xw1 = nb((qk > 0 && pk + 1 < np) ? -d : 0, 0);
    const float2 xw2 = nb(0, (pl > 0 && ql + 1 < nq) ? d : 0);
    const float ur = fmaf(-u2, xu2.x, u1 * xu1.x), ui = fmaf(-u2, xu2.y, u1 * xu1.y);
    const float wr = fmaf(-w2, xw2.x, w1 * xw1.x), wi = fmaf(-w2, xw2.y, w1 * xw1.y);
    const float2 c = S.ctf[H.Q + kp];
    const float a = ADJ ? -c.x : c.x, b = ADJ ? -c.y : c.y;
    ar = fmaf(b, ur - wr, fmaf(a, ui + wi, ar));
    ai = fmaf(b, ui - wi, fmaf(-a, ur + wr, ai));
  }
}

// ---------------------------------------------------------------------------
// Paired-single apply (lb_set_precision LB_PREC_F32X2).  A value is a pair
// (hi, lo) of single-precision numbers; acc += (ch + cl)(xh + xl) forms the
// product ch xh with its exact rounding error (one FMA), adds the cross terms
// ch xl + cl xh to that error (cl xl, below 2^-48 of the product, is
// dropped), and adds ch xh to the running hi part with its exact rounding
// error (two-sum), which goes to the lo part with the product's error.  The
// _rn intrinsics keep the compiler from contracting these steps.
__device__ __forceinline__ void ffmac(float& sh, float& sl, float ch, float cl, float xh, float xl) {
  const float p = __fmul_rn(ch, xh);
  float e = __fmaf_rn(ch, xh, -p);
  e = __fmaf_rn(ch, xl, e);
  e = __fmaf_rn(cl, xh, e);
  const float sum = __fadd_rn(sh, p);
  const float bv = __fsub_rn(sum, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(sum, bv)), __fsub_rn(p, bv));
  sh = sum;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}
// (ph, pe) = (ah + al)(bh + bl): the product of the hi parts with its exact
// rounding error and the cross terms (an unnormalised pair)
__device__ __forceinline__ float2 ffprod(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  return make_float2(p, e);
}
// (ah + al) + (bh + bl): two-sum of the hi parts, the lo parts and the
// two-sum's error added in single precision (an unnormalised pair)
__device__ __forceinline__ float2 ffadd(float2 a, float2 b) {
  const float sum = __fadd_rn(a.x, b.x);
  const float bv = __fsub_rn(sum, a.x);
  const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(sum, bv)), __fsub_rn(b.x, bv));
  return make_float2(sum, __fadd_rn(__fadd_rn(a.y, b.y), t));
}
__device__ __forceinline__ float2 ffneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float4 split4(double2 z) {
  const float2 a = split_f64(z.x), b = split_f64(z.y);
  return make_float4(a.x, a.y, b.x, b.y);
}
// entry (k, l) of a packed Hermitian split iterate (x_hi, x_lo, y_hi, y_lo)
__device__ __forceinline__ float4 ldpk4(const float4* p, int k, int l) {
  const bool lo = k > l;
  const int a = lo ? l : k, c = lo ? k : l;
  const float4* q = p + ((c * (c + 1)) >> 1) + a;
  float4 x = kNbL2 ? __ldcg(q) : *q;
  const unsigned f = lo ? 0x80000000u : 0u;
  x.z = __uint_as_float(__float_as_uint(x.z) ^ f);
  x.w = __uint_as_float(__float_as_uint(x.w) ^ f);
  return x;
}

// offdiag_acc on a split iterate in paired single precision: acc = (re hi,
// re lo, im hi, im lo) of the control and decay terms, the same sums as
// offdiag_acc with the pairs of S.ffcu, S.ffcd, S.ffab and S.ffjf / S.ffja.
// No Jaynes-Cummings pairs.
template <bool ADJ, bool PK, int QN>
__device__ __forceinline__ void offdiag_acc_ff(float (&acc)[4], const float4* __restrict__ x, int v, uint32_t kd,
                                               uint32_t ld, const Hdr& H, const GridSmem& S, int k, int l) {
  const int N = H.N;
  auto nb = [&](int dk, int dl) -> float4 {
    if constexpr (PK) {
      return ldpk4(x, k + dk, l + dl);
    } else {
      const float4* q = x + v + dk + dl * N;
      return kNbL2 ? __ldcg(q) : *q;
    }
  };
  auto sub = [&](int q) {
    const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
    const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
    // the ladder factors c1 = cu[nk], c2 = cd[nl], c3 = cd[nk], c4 = cu[nl]
    // as pairs; P = c1 x1 - c2 x2, R = c3 x3 - c4 x4 and, with this solve's
    // (a, b) (negated for the adjoint), re += b (P - R)_re + a (P + R)_im,
    // im += b (P - R)_im - a (P + R)_re, as in offdiag_acc
    const float2 c1 = S.ffcu[co + nk], c2 = S.ffcd[co + nl], c3 = S.ffcd[co + nk], c4 = S.ffcu[co + nl];
    const float4 x1 = nb(nk + 1 < n ? s : 0, 0);
    const float4 x2 = nb(0, nl > 0 ? -s : 0);
    const float4 x3 = nb(nk > 0 ? -s : 0, 0);
    const float4 x4 = nb(0, nl + 1 < n ? s : 0);
    const float2 pr = ffadd(ffprod(c1.x, c1.y, x1.x, x1.y), ffprod(-c2.x, -c2.y, x2.x, x2.y));
    const float2 pi = ffadd(ffprod(c1.x, c1.y, x1.z, x1.w), ffprod(-c2.x, -c2.y, x2.z, x2.w));
    const float2 rr = ffadd(ffprod(c3.x, c3.y, x3.x, x3.y), ffprod(-c4.x, -c4.y, x4.x, x4.y));
    const float2 ri = ffadd(ffprod(c3.x, c3.y, x3.z, x3.w), ffprod(-c4.x, -c4.y, x4.z, x4.w));
    const float2 ur = ffadd(pr, rr), ui = ffadd(pi, ri), wr = ffadd(pr, ffneg(rr)), wi = ffadd(pi, ffneg(ri));
    const float4 ab = S.ffab[q];  // (b hi, b lo, a hi, a lo)
    ffmac(acc[0], acc[1], ab.x, ab.y, wr.x, wr.y);
    ffmac(acc[0], acc[1], ab.z, ab.w, ui.x, ui.y);
    ffmac(acc[2], acc[3], ab.x, ab.y, wi.x, wi.y);
    ffmac(acc[2], acc[3], -ab.z, -ab.w, ur.x, ur.y);
    if ((H.jon >> q) & 1u) {
      const int jo = H.joff[q] + nk * n + nl;
      float2 cj;
      float4 x5;
      if (!ADJ) {
        cj = S.ffjf[jo];
        const int d = (nk + 1 < n && nl + 1 < n) ? s : 0;
        x5 = nb(d, d);
      } else {
        cj = S.ffja[jo];
        const int d = (nk > 0 && nl > 0) ? s : 0;
        x5 = nb(-d, -d);
      }
      ffmac(acc[0], acc[1], cj.x, cj.y, x5.x, x5.y);
      ffmac(acc[2], acc[3], cj.x, cj.y, x5.z, x5.w);
    }
  };
  if constexpr (QN > 0) {
#pragma unroll
    for (int q = 0; q < QN; ++q) sub(q);
  } else {
    for (int q = 0; q < H.Q; ++q) sub(q);
  }
}

// One difference iteration over a block's chunk [e0, e1): from the change dc
// of the last iteration (single precision), the new iterate zn = zc + its
// change dn, the FP64 correction in cring (the predictor's ring slot, when
// the solve records one) updated, and the per-state maxima of the change
// pushed to `bank`.
template <bool ADJ, int QN>
__device__ __forceinline__ void grid_diff_pass(const ProbDev& P, const GridSmem& S, long long e0, long long e1,
                                            const float2* __restrict__ dc, float2* __restrict__ dn,
                                            const double2* __restrict__ zc, double2* __restrict__ zn,
                                            float4* __restrict__ zsn, double2* __restrict__ cring,
                                            unsigned long long* bank) {
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  StateMax sm;
  sm.init(e0, e1, G.Vh);
  for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
    const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
    const int b = g.b, v = g.v;
    const size_t o = gslab(G, g, b);
    const uint32_t kd = __ldg(P.digits + g.k), ld = __ldg(P.digits + g.l);
    // (dt/2) O d in single precision: the change of the correction
    float fr = 0.0f, fi = 0.0f;
    if (G.herm)
      offdiag_acc_f<ADJ, true, QN>(fr, fi, dc + (size_t)b * G.Vh, v, kd, ld, H, S, g.k, g.l);
    else
      offdiag_acc_f<ADJ, false, QN>(fr, fi, dc + (size_t)b * G.Vh, v, kd, ld, H, S, g.k, g.l);
    if (cring) {
      const double2 c = cring[o];
      cring[o] = make_double2(c.x + f32_to_f64(fr), c.y + f32_to_f64(fi));
    }
    // the change of the iterate, (I - dt/2 D)^-1 times that
    const float2 df = __ldg(P.Dinvf + v);
    const float dfi = ADJ ? -df.y : df.y;
    const float ex = fmaf(df.x, fr, -dfi * fi), ey = fmaf(df.x, fi, dfi * fr);
    const double ddx = f32_to_f64(ex), ddy = f32_to_f64(ey);
    const double2 zo = __ldcg(zc + o);
    const double2 z = make_double2(zo.x + ddx, zo.y + ddy);
    zn[o] = z;
    if (zsn) zsn[o] = split4(z);
    dn[o] = make_float2(ex, ey);
    sm.add(b, umax64(abs_bits(ddx), abs_bits(ddy)), bank);
  }
  sm.push(bank, reinterpret_cast<unsigned long long*>(S.red));
}

// One FP64 Jacobi (or Neumann) iteration over a block's chunk [e0, e1): the
// correction (dt/2) O z of the iterate zc, kept apart from the right-hand
// side (with the predictor on it goes to the ring slot cring of this step;
// the last iteration's write stays: the correction whose Jacobi image is the
// returned z), the new iterate zn, its single-precision change dnew (for a
// difference iteration next) and the per-state maxima of the change pushed
// to `bank`.  QN: the subsystem count at compile time (0: H.Q at run time).
template <bool ADJ, int QN, bool FF>
__device__ __forceinline__ void grid_full_pass(const ProbDev& P, const GridSmem& S, long long e0, long long e1,
                                            const double2* __restrict__ rhs, const double2* __restrict__ ct,
                                            const double2* __restrict__ zc, double2* __restrict__ zn,
                                            const float4* __restrict__ zsc, float4* __restrict__ zsn,
                                            double2* __restrict__ cring, float2* __restrict__ dnew, bool neumann,
                                            double hh, unsigned long long* bank) {
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  StateMax sm;
  sm.init(e0, e1, G.Vh);
  for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
    const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
    const int b = g.b, v = g.v;
    const double2* xs = zc + (size_t)b * G.Vh;
    const size_t o = gslab(G, g, b);
    const double2 r = rhs[o];
    double cr = 0.0, ci = 0.0;
    const uint32_t kd = __ldg(P.digits + g.k), ld = __ldg(P.digits + g.l);
    if constexpr (FF) {
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (G.herm)
        offdiag_acc_ff<ADJ, true, QN>(acc, zsc + (size_t)b * G.Vh, v, kd, ld, H, S, g.k, g.l);
      else
        offdiag_acc_ff<ADJ, false, QN>(acc, zsc + (size_t)b * G.Vh, v, kd, ld, H, S, g.k, g.l);
      cr = f32_to_f64(acc[0]) + f32_to_f64(acc[1]);
      ci = f32_to_f64(acc[2]) + f32_to_f64(acc[3]);
    } else {
      if (G.herm)
        offdiag_acc<ADJ, kNbL2, true, QN>(cr, ci, xs, v, kd, ld, H, T, ct, g.k, g.l);
      else
        offdiag_acc<ADJ, kNbL2, false, QN>(cr, ci, xs, v, kd, ld, H, T, ct);
    }
    if (cring) cring[o] = make_double2(cr, ci);
    const double ar = r.x + cr, ai = r.y + ci;
    const double2 zo = __ldcg(xs + g.i);
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
    zn[o] = z;
    if constexpr (FF) zsn[o] = split4(z);
    const double ddx = z.x - zo.x, ddy = z.y - zo.y;
    if (dnew) dnew[o] = make_float2(f64_to_f32_trunc(ddx), f64_to_f32_trunc(ddy));
    sm.add(b, umax64(abs_bits(ddx), abs_bits(ddy)), bank);
  }
  sm.push(bank, reinterpret_cast<unsigned long long*>(S.red));
}

// The first pass of a solve, per element g (slab offset o, right-hand side
// r): z_0 = (I - dt/2 D)^-1 (r + the predicted correction) for the Jacobi
// iteration (r itself for the Neumann series) into zA (and its split, FF),
// |r| into the solve's per-state maxima and, with the running penalty
// (pen), the merit summand of r into msum.
template <bool ADJ, bool FF>
__device__ __forceinline__ void first_elem(const ProbDev& P, const GridHdr& G, const GEl& g, size_t o, double2 r,
                                           const GridHist& hist, bool pen, bool neumann,
                                           double (&msum)[kLocalStates], StateMax& sm, unsigned long long* qbank) {
  const Hdr& H = G.h;
  const int b = g.b, v = g.v;
  if (pen) {
    // an off-diagonal element under the symmetry stands for its mirror too
    const double f = merit_summand(H.kind, r, P.tar[(size_t)b * H.V + v]) * (g.vm >= 0 ? 2.0 : 1.0);
    const int k = b - sm.sb0;
#pragma unroll
    for (int u = 0; u < kLocalStates; ++u)
      if (u == k) msum[u] += f;
  }
  double2 z0 = r;
  if (!neumann) {
    double ur = r.x, ui = r.y;
    const double2 d = __ldg(P.Dinv + v);
    const double di = ADJ ? -d.y : d.y;
    if (hist.n > 0) {
      const double2 c = cmul(hist.gp[o], anchored_sum(hist.ring + o, (size_t)G.M * G.Vh, hist.slot, hist.n));
      ur += c.x;
      ui += c.y;
    } else if (hist.ring) {
      // a fresh anchor: m = 0
      hist.gp[o] = make_double2(1.0, 0.0);
      hist.gm[o] = make_double2(1.0, 0.0);
    }
    z0 = make_double2(fma(d.x, ur, -di * ui), fma(d.x, ui, di * ur));
  }
  P.zA[o] = z0;
  if constexpr (FF) P.zsA[o] = split4(z0);
  sm.add(b, umax64(abs_bits(r.x), abs_bits(r.y)), qbank);
}
// ... and per block, after the elements (all threads): push the maxima and,
// with the running penalty, the block's merit sums of its chunk's states in
// a fixed order
__device__ __forceinline__ void first_end(const ProbDev& P, const GridSmem& S, StateMax& sm,
                                          unsigned long long* qbank, bool pen, const double (&msum)[kLocalStates]) {
  sm.push(qbank, reinterpret_cast<unsigned long long*>(S.red));
  if (pen) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double* dred = S.red;
#pragma unroll
    for (int u = 0; u < kLocalStates; ++u) {
      const double w = warp_sum(msum[u]);
      if (lane == 0) dred[u * 8 + warp] = w;
    }
    __syncthreads();
    if ((int)threadIdx.x < kLocalStates) {
      double t = 0.0;
      for (int w = 0; w < nwarps; ++w) t += dred[threadIdx.x * 8 + w];
      P.mpart[(size_t)blockIdx.x * kLocalStates + threadIdx.x] = t;
    }
    __syncthreads();
  }
}

// One implicit-midpoint solve over all M states (see above).  prepped: the
// first pass was already done by the caller (first_elem / first_end, fused
// with the previous step's commit), for this solve's |q| bank.
template <bool ADJ, bool FF>
__device__ int grid_solve(const ProbDev& P, const GridSmem& S, const double2* __restrict__ rhs,
                          const double2* __restrict__ ct, double fac, long long& it_global, long long& solve,
                          int& ndiff, double2** zout, GridHist hist = GridHist(), double penw = 0.0,
                          bool prepped = false) {
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const Tabs T{S.cu, S.cd, S.jf, S.ja};
  const bool neumann = H.method == LB_SOLVER_NEUMANN;
  const int M = G.M, V = H.V;
  const long long e0 = (long long)blockIdx.x * G.chunk;
  const long long e1 = min(G.total, e0 + G.chunk);
  unsigned long long* dslots = P.gslots;          // [3][M]
  unsigned long long* qslots = P.gslots + 3 * M;  // [2][M]
  unsigned long long* qbank = qslots + (solve & 1) * M;
  unsigned long long* red = reinterpret_cast<unsigned long long*>(S.red);
  // difference iterations: Jacobi only; this solve's control factors in single precision
  const bool dok = P.diffit && !neumann && P.dfA != nullptr;
  if (dok && (int)threadIdx.x < H.cq) S.ctf[threadIdx.x] = make_float2((float)ct[threadIdx.x].x, (float)ct[threadIdx.x].y);
  // paired-single apply: this solve's factor tables (the adjoint's with -a, -b)
  constexpr bool ff = FF;
  if (ff && (int)threadIdx.x < H.Q) {
    const int q = threadIdx.x;
    const float2 a = split_f64(ADJ ? -ct[q].x : ct[q].x), b = split_f64(ADJ ? -ct[q].y : ct[q].y);
    S.ffab[q] = make_float4(b.x, b.y, a.x, a.y);
  }
  ndiff = 0;
  // z_0 = (I - dt/2 D)^-1 rhs (Jacobi) or rhs (Neumann); per-state max |rhs|
  if (!prepped) {
    StateMax sm;
    sm.init(e0, e1, G.Vh);
    double msum[kLocalStates] = {0.0, 0.0, 0.0, 0.0};
    for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
      const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
      const size_t o = gslab(G, g, g.b);
      first_elem<ADJ, FF>(P, G, g, o, rhs[o], hist, penw != 0.0, neumann, msum, sm, qbank);
    }
    first_end(P, S, sm, qbank, penw != 0.0, msum);
  }
  if (!grid_sync(P.bar, gridDim.x, P.spin_limit > 0 ? P.spin_limit : kSpinLimit)) return -3;
  if (penw != 0.0 && blockIdx.x == 0) {
    // state b's merit sum over the blocks whose chunk covers it, in block order
    for (int b = threadIdx.x; b < M; b += blockDim.x) {
      double t = 0.0;
      for (int bb = 0; bb < (int)gridDim.x; ++bb) {
        const long long f0 = (long long)bb * G.chunk, f1 = min(G.total, f0 + G.chunk);
        if (f0 >= f1) break;
        const int s0 = (int)(f0 / G.Vh), s1 = (int)((f1 - 1) / G.Vh);
        if (b >= s0 && b <= s1) t += __ldcg(P.mpart + (size_t)bb * kLocalStates + (b - s0));
      }
      P.jpen[b] = fma(penw, merit_value(H.kind, t), P.jpen[b]);
    }
  }
  // the previous solve's |q| bank is free again: clear it for the next solve
  if (blockIdx.x == 0)
    for (int b = threadIdx.x; b < M; b += blockDim.x) qslots[((solve + 1) & 1) * M + b] = 0;
  ++solve;
  const double hh = 0.5 * H.h;
  double2* zc = P.zA;
  double2* zn = P.zB;
  // single-precision changes of the iterates: iteration `it` writes the
  // change of zn to dfB (even it) or dfA (odd it) and a difference iteration
  // reads the other buffer
  bool dit = false;  // this iteration is a difference iteration
  for (int it = 0; it < H.max_iter; ++it, ++it_global) {
    unsigned long long* bank = dslots + (it_global % 3) * M;
    if (dit) {
      ++ndiff;
      const float2* dcur = (it & 1) ? P.dfB : P.dfA;
      float2* dnew = (it & 1) ? P.dfA : P.dfB;
      float4* zsdn = ff ? ((it & 1) ? P.zsA : P.zsB) : nullptr;
      double2* cring = hist.ring ? hist.ring + (size_t)hist.slot * ((size_t)M * G.Vh) : nullptr;
      switch (H.Q) {
        case 1: grid_diff_pass<ADJ, 1>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 2: grid_diff_pass<ADJ, 2>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 3: grid_diff_pass<ADJ, 3>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 4: grid_diff_pass<ADJ, 4>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 5: grid_diff_pass<ADJ, 5>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 6: grid_diff_pass<ADJ, 6>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        case 7: grid_diff_pass<ADJ, 7>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
        default: grid_diff_pass<ADJ, 8>(P, S, e0, e1, dcur, dnew, zc, zn, zsdn, cring, bank); break;
      }
    } else {
      double2* cring = hist.ring ? hist.ring + (size_t)hist.slot * ((size_t)M * G.Vh) : nullptr;
      float2* dnew = dok ? ((it & 1) ? P.dfA : P.dfB) : nullptr;
      // the subsystem counts of the large workloads (4 and 6) get an
      // unrolled subsystem loop; other counts run the general loop
      if constexpr (ff) {
        const float4* zsc = (it & 1) ? P.zsB : P.zsA;
        float4* zsn = (it & 1) ? P.zsA : P.zsB;
        switch (H.Q) {
          case 4: grid_full_pass<ADJ, 4, true>(P, S, e0, e1, rhs, ct, zc, zn, zsc, zsn, cring, dnew, neumann, hh, bank); break;
          case 6: grid_full_pass<ADJ, 6, true>(P, S, e0, e1, rhs, ct, zc, zn, zsc, zsn, cring, dnew, neumann, hh, bank); break;
          default: grid_full_pass<ADJ, 0, true>(P, S, e0, e1, rhs, ct, zc, zn, zsc, zsn, cring, dnew, neumann, hh, bank); break;
        }
      } else {
        switch (H.Q) {
          case 4: grid_full_pass<ADJ, 4, false>(P, S, e0, e1, rhs, ct, zc, zn, nullptr, nullptr, cring, dnew, neumann, hh, bank); break;
          case 6: grid_full_pass<ADJ, 6, false>(P, S, e0, e1, rhs, ct, zc, zn, nullptr, nullptr, cring, dnew, neumann, hh, bank); break;
          default: grid_full_pass<ADJ, 0, false>(P, S, e0, e1, rhs, ct, zc, zn, nullptr, nullptr, cring, dnew, neumann, hh, bank); break;
        }
      }
    }
    if (!grid_sync(P.bar, gridDim.x, P.spin_limit > 0 ? P.spin_limit : kSpinLimit)) return -3;
    // bank of iteration it_global + 2 is no longer read by anyone: clear it
    if (blockIdx.x == 0)
      for (int b = threadIdx.x; b < M; b += blockDim.x) dslots[((it_global + 2) % 3) * M + b] = 0;
    // every block takes the same decision from the same slots (the states
    // spread over the lanes of warp 0)
    if (threadIdx.x < 32) {
      bool bad = false, open = false, small = true;
      for (int b = threadIdx.x; b < M; b += 32) {
        const unsigned long long d = __ldcg(bank + b);
        const unsigned long long q = __ldcg(qbank + b);
        if (d >= kInfBits || q >= kInfBits) {
          bad = true;
        } else {
          const double qd = __longlong_as_double((long long)q);
          const unsigned long long thr = abs_bits(H.rtol * qd * fac);
          if (d > thr) open = true;
          // a difference iteration next: every state's change below kDiffRel max|q|
          if (!(qd >= kDiffFloor) || d > abs_bits(kDiffRel * qd)) small = false;
        }
      }
      bad = __any_sync(kFull, bad);
      open = __any_sync(kFull, open);
      small = __all_sync(kFull, small);
      if (threadIdx.x == 0) {
        S.flag[0] = bad ? -2 : (open ? 0 : 1);  // NaN/Inf, not yet, converged
        S.flag[1] = dok && small ? 1 : 0;
      }
    }
    __syncthreads();
    const int state = S.flag[0];
    dit = S.flag[1] != 0;
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
// Blocks per SM the grid kernels are compiled for (registers per thread:
// 128 at 2 blocks of 256 threads, 85 at 3).  Measured: three blocks (24
// warps per SM) make the paired-single kernels 8 % faster on workload 5
// (vec 531441, 64 states) despite their spills to local memory, whose load
// latency the extra warps hide; the FP64 kernels gain under 1 % there and
// lose 2-4 % on the smaller grid workloads (vec 65536 and 6400, a few
// states), where more blocks only lengthen each grid barrier, so they keep
// two.
constexpr int kBlocksPerSM64 = 2;
constexpr int kBlocksPerSMFF = 3;

// FF: the FP64 iterations apply O in paired single precision (P.ff); the
// two variants are separate kernels so that each has its own registers
template <bool FF>
__global__ void __launch_bounds__(kGridThreads, FF ? kBlocksPerSMFF : kBlocksPerSM64) k_sweep_grid(const ProbDev* __restrict__ pp, int mode, int init,
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
  // the running state: the system's own states in the sweep buffer qf (its
  // slab layout), or the caller's vectors (vec layout, no symmetry)
  double2* q = mode == 0 ? P.qf : x;
  const long long e0 = (long long)blockIdx.x * G.chunk, e1 = min(G.total, e0 + G.chunk);
  if (mode == 0)
    for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
      const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
      q[gslab(G, g, g.b)] = (init ? P.q0 : P.qT)[(size_t)g.b * V + g.v];
    }
  bool failed = false;
  long long itg = 0, nsolve = 0;
  unsigned long long iters = 0, steps = 0, diters = 0;
  int maxit = 0;
  const int phase = mode == 2 ? 2 : 0;
  // first-iterate predictor of the forward sweep, forgetting its history at
  // every step j with j % R == 0 (R > 0 divides K, so every checkpoint is a
  // restart point and the recompute repeats these iterates bit for bit)
  const int R = P.pred_restart;
  const bool pred = mode == 0 && R >= 0;
  // the running penalty is summed over the forward sweep of the system's own states
  const bool penal = mode == 0 && H.gamma1 != 0.0;
  GridHist hist;
  hist.ring = P.hist;
  hist.gp = P.hgp;
  hist.gm = P.hgm;
  hist.cap = P.pred_order;
  const bool neumann = H.method == LB_SOLVER_NEUMANN;
  bool prepped = false;  // this step's first pass was fused with the previous step's commit
  for (int jj = 0; jj < j1 - j0; ++jj) {
    const int j = mode == 2 ? j1 - 1 - jj : j0 + jj;
    if (!prepped) {
      if (pred && R > 0 && j % R == 0) hist.restart();
      if (mode == 0 && tape && H.K > 0 && j % H.K == 0) {
        for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
          const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
          P.ckpt[gslab(G, g, (size_t)g.b * H.n_ckpt + j / H.K)] = q[gslab(G, g, g.b)];
        }
      }
    }
    double2* z = nullptr;
    int nd = 0;
    const int it = mode == 2 ? grid_solve<true, FF>(P, S, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve,
                                                nd, &z, GridHist(), 0.0, prepped)
                             : grid_solve<false, FF>(P, S, q, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve,
                                                 nd, &z, pred ? hist : GridHist(), penal ? P.pen[j] : 0.0, prepped);
    if (it < 0) {
      grid_fail(P, it, j);
      failed = true;
      break;
    }
    iters += (unsigned long long)it * G.M;
    diters += (unsigned long long)nd * G.M;
    steps += G.M;
    maxit = max(maxit, it);
    // this step's commit (q^{j+1} = 2 z - q^j, the predictor's record), in
    // the same pass as the first pass of the next step (its predictor state
    // hn: advanced, restarted where the next step is a restart point)
    // (the adjoint propagation of mode 2 keeps separate passes)
    const bool next = mode != 2 && jj + 1 < j1 - j0;
    const int jn = j + 1;
    GridHist hn = hist;
    if (pred) {
      hn.advance();
      if (hn.m >= kAnchorSteps) hn.m = 0;
      if (next && R > 0 && jn % R == 0) hn.restart();
    }
    const bool ckn = next && mode == 0 && tape && H.K > 0 && jn % H.K == 0;
    const bool penn = next && penal && P.pen[jn] != 0.0;
    unsigned long long* qbn = P.gslots + 3 * G.M + (nsolve & 1) * G.M;  // the next solve's |q| bank
    StateMax smn;
    smn.init(e0, e1, G.Vh);
    double msum[kLocalStates] = {0.0, 0.0, 0.0, 0.0};
    for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
      const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
      const size_t o = gslab(G, g, g.b);
      const double2 zz = z[o], qq = q[o];
      if (mode == 0 && tape && H.K == 0) P.ckpt[gslab(G, g, (size_t)g.b * H.NT + j)] = zz;
      const double2 qn = make_double2(fma(2.0, zz.x, -qq.x), fma(2.0, zz.y, -qq.y));
      q[o] = qn;
      if (pred) grid_commit<false>(P, hist, o, (size_t)G.M * G.Vh, g.v);
      if (next) {
        if (ckn) P.ckpt[gslab(G, g, (size_t)g.b * H.n_ckpt + jn / H.K)] = qn;
        first_elem<false, FF>(P, G, g, o, qn, pred ? hn : GridHist(), penn, neumann, msum, smn, qbn);
      }
    }
    if (next) first_end(P, S, smn, qbn, penn, msum);
    if (pred) hist = hn;
    prepped = next;
  }
  // the final states rho_i(T), in the vec layout with their mirrors
  if (mode == 0 && !failed)
    for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
      const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
      gput(P.qT, g, V, q[gslab(G, g, g.b)]);
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&P.status->iters[phase], iters);
    atomicAdd(&P.status->steps[phase], steps);
    atomicAdd(&P.status->diters[phase], diters);
    atomicMax(&P.status->max_iter_seen, maxit);
  }
}

// backward sweep over all states: recompute each checkpoint segment, then the
// adjoint steps with the gradient pieces summed over states and blocks
template <bool FF>
__global__ void __launch_bounds__(kGridThreads, FF ? kBlocksPerSMFF : kBlocksPerSM64)
    k_backward_grid(const ProbDev* __restrict__ pp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const ProbDev& P = *pp;
  const GridSmem S = grid_setup(smem, P, P.M, P.herm);
  const GridHdr& G = *S.g;
  const Hdr& H = G.h;
  const int V = H.V, N = H.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const long long e0 = (long long)blockIdx.x * G.chunk, e1 = min(G.total, e0 + G.chunk);
  // terminal condition qhat^{N_T} = beta_i/M g_i (Appendix B)
  for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
    const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
    const size_t o = (size_t)g.b * V + g.v;
    const double w = P.wgt[g.b];
    const double wt = linear_sign(P.kind) * w;
    const double2 t = P.tar[o];
    if (H.kind == LB_J_FROB) {
      const double2 qq = P.qT[o];
      P.lam[gslab(G, g, g.b)] = make_double2(w * (qq.x - t.x), w * (qq.y - t.y));
    } else {
      P.lam[gslab(G, g, g.b)] = make_double2(wt * t.x, wt * t.y);
    }
  }
  // running penalty: q^j is rebuilt backwards, q^j = 2 z^j - q^{j+1}, in
  // P.qb (each element by its own thread), from q^{N_T}
  const bool penal = H.gamma1 != 0.0;
  if (penal)
    for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
      const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
      P.qb[gslab(G, g, g.b)] = P.qT[(size_t)g.b * V + g.v];
    }
  long long itg = 0, nsolve = 0;
  unsigned long long it_rec = 0, st_rec = 0, it_adj = 0, st_adj = 0, dit_rec = 0, dit_adj = 0;
  int maxit = 0;
  const int nseg = H.K > 0 ? (H.NT + H.K - 1) / H.K : 1;
  bool failed = false;
  // adjoint predictor: the adjoint steps come in the same order for every K
  const bool apred = H.method != LB_SOLVER_NEUMANN;
  GridHist ahist;
  ahist.ring = P.hist;
  ahist.gp = P.hgp;
  ahist.gm = P.hgm;
  ahist.cap = P.pred_order;
  // forward predictor of the recompute, restarted as in the forward sweep
  const int R = P.pred_restart;
  const bool fpred = H.K > 0 && R > 0;
  GridHist fhist;
  fhist.ring = P.histf;
  fhist.gp = P.fgp;
  fhist.gm = P.fgm;
  fhist.cap = P.pred_order;
  for (int sg = nseg - 1; sg >= 0 && !failed; --sg) {
    const int j0 = H.K > 0 ? sg * H.K : 0;
    const int j1 = H.K > 0 ? min(H.NT, j0 + H.K) : H.NT;
    if (H.K > 0) {
      for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
        const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
        P.qf[gslab(G, g, g.b)] = P.ckpt[gslab(G, g, (size_t)g.b * H.n_ckpt + sg)];
      }
      for (int j = j0; j < j1; ++j) {
        double2* z = nullptr;
        if (fpred && j % R == 0) fhist.restart();  // every checkpoint is a restart point
        int nd = 0;
        const int it = grid_solve<false, FF>(P, S, P.qf, P.ctab + (size_t)j * H.cq, stop_factor(P, j), itg, nsolve, nd,
                                         &z, fpred ? fhist : GridHist());
        if (it < 0) {
          grid_fail(P, it, j);
          failed = true;
          break;
        }
        it_rec += (unsigned long long)it * G.M;
        dit_rec += (unsigned long long)nd * G.M;
        st_rec += G.M;
        maxit = max(maxit, it);
        for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
          const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
          const size_t o = gslab(G, g, g.b);
          const double2 zz = z[o], qq = P.qf[o];
          P.seg[gslab(G, g, (size_t)g.b * H.K + (j - j0))] = zz;  // read back at the same element only
          P.qf[o] = make_double2(fma(2.0, zz.x, -qq.x), fma(2.0, zz.y, -qq.y));
          if (fpred) grid_commit<false>(P, fhist, o, (size_t)G.M * G.Vh, g.v);
        }
        if (fpred) {
          fhist.advance();
          if (fhist.m >= kAnchorSteps) fhist.m = 0;
        }
      }
      if (failed) break;
    }
    for (int j = j1 - 1; j >= j0; --j) {
      const double2* ct = P.ctab + (size_t)j * H.cq;
      double2* zh = nullptr;
      int nd = 0;
      const int it =
          grid_solve<true, FF>(P, S, P.lam, ct, stop_factor(P, j), itg, nsolve, nd, &zh, apred ? ahist : GridHist());
      if (it < 0) {
        grid_fail(P, it, j);
        failed = true;
        break;
      }
      it_adj += (unsigned long long)it * G.M;
      dit_adj += (unsigned long long)nd * G.M;
      st_adj += G.M;
      maxit = max(maxit, it);
      // Passes over this block's elements, four subsystems each (so that the
      // sums stay in registers): the gradient pieces (eq. reducedgradient),
      // summed per block, and in the last pass the update
      // qhat^j = 2 zhat - qhat^{j+1} with the predictor's record.
      //   g_a  = -i sum_kl Z_kl conj(R_zhat),  g_ad = -i sum_kl Z_kl conj(P_zhat)
      // with P, R the neighbour combinations of offdiag_acc taken on zhat.
      constexpr int kQP = 4;  // subsystems per pass
      const int Qn = H.Q;
      for (int q0 = 0; q0 < Qn; q0 += kQP) {
        const bool last = q0 + kQP >= Qn;
        double sar[kQP], sai[kQP], sdr[kQP], sdi[kQP];
#pragma unroll
        for (int u = 0; u < kQP; ++u) sar[u] = sai[u] = sdr[u] = sdi[u] = 0.0;
        // paired-single sums (FF): (g_a re hi, lo, im hi, lo), (g_ad ...)
        float fa[kQP][4], fb[kQP][4];
#pragma unroll
        for (int u = 0; u < kQP; ++u)
#pragma unroll
          for (int c = 0; c < 4; ++c) fa[u][c] = fb[u][c] = 0.0f;
        // zhat split into pairs: the buffer the solve's last iteration wrote
        const float4* zsh = FF ? (zh == P.zA ? P.zsA : P.zsB) : nullptr;
        for (GIter it_(G, e0 + threadIdx.x); it_.e < e1; it_.next(G, blockDim.x)) {
          const GEl g = gel_at(G, P.hkl, it_.b, it_.i);
          const int b = g.b, v = g.v;
          const size_t o = gslab(G, g, b);
          const double2* zs = zh + (size_t)b * G.Vh;
          const double2 Z = H.K > 0 ? P.seg[gslab(G, g, (size_t)b * H.K + (j - j0))]
                                    : P.ckpt[gslab(G, g, (size_t)b * H.NT + j)];
          const uint32_t kd = __ldg(P.digits + g.k), ld = __ldg(P.digits + g.l);
          // entry at row offset dk, column offset dl of zhat (packed under the symmetry)
          auto nb = [&](int dk, int dl) -> double2 {
            return G.herm ? ldpk<kNbL2>(zs, g.k + dk, g.l + dl) : ldz<kNbL2>(zs + v + dk + dl * N);
          };
          if constexpr (FF) {
            // the same pieces in paired single precision from the split zhat
            const float4* zss = zsh + (size_t)b * G.Vh;
            auto nbf = [&](int dk, int dl) -> float4 {
              if (G.herm) return ldpk4(zss, g.k + dk, g.l + dl);
              const float4* qq = zss + v + dk + dl * N;
              return kNbL2 ? __ldcg(qq) : *qq;
            };
            const float4 Zs = split4(Z);
#pragma unroll
            for (int u = 0; u < kQP; ++u) {
              const int q = q0 + u;
              if (q < Qn) {
                const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
                const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
                const float2 c1 = S.ffcu[co + nk], c2 = S.ffcd[co + nl], c3 = S.ffcd[co + nk], c4 = S.ffcu[co + nl];
                const float4 x1 = nbf(nk + 1 < n ? s : 0, 0);
                const float4 x2 = nbf(0, nl > 0 ? -s : 0);
                const float4 x3 = nbf(nk > 0 ? -s : 0, 0);
                const float4 x4 = nbf(0, nl + 1 < n ? s : 0);
                const float2 pr = ffadd(ffprod(c1.x, c1.y, x1.x, x1.y), ffprod(-c2.x, -c2.y, x2.x, x2.y));
                const float2 pi = ffadd(ffprod(c1.x, c1.y, x1.z, x1.w), ffprod(-c2.x, -c2.y, x2.z, x2.w));
                const float2 rr = ffadd(ffprod(c3.x, c3.y, x3.x, x3.y), ffprod(-c4.x, -c4.y, x4.x, x4.y));
                const float2 ri = ffadd(ffprod(c3.x, c3.y, x3.z, x3.w), ffprod(-c4.x, -c4.y, x4.z, x4.w));
                if (G.herm && g.vm >= 0) {
                  const float2 dr = ffadd(rr, ffneg(pr)), di = ffadd(ri, ffneg(pi));
                  const float2 ur = ffadd(rr, pr), ui = ffadd(ri, pi);
                  ffmac(fa[u][0], fa[u][1], Zs.x, Zs.y, dr.x, dr.y);
                  ffmac(fa[u][0], fa[u][1], Zs.z, Zs.w, di.x, di.y);
                  ffmac(fa[u][2], fa[u][3], Zs.z, Zs.w, ur.x, ur.y);
                  ffmac(fa[u][2], fa[u][3], -Zs.x, -Zs.y, ui.x, ui.y);
                } else {
                  ffmac(fa[u][0], fa[u][1], Zs.x, Zs.y, rr.x, rr.y);
                  ffmac(fa[u][0], fa[u][1], Zs.z, Zs.w, ri.x, ri.y);
                  ffmac(fa[u][2], fa[u][3], Zs.z, Zs.w, rr.x, rr.y);
                  ffmac(fa[u][2], fa[u][3], -Zs.x, -Zs.y, ri.x, ri.y);
                  if (!G.herm) {
                    ffmac(fb[u][0], fb[u][1], Zs.x, Zs.y, pr.x, pr.y);
                    ffmac(fb[u][0], fb[u][1], Zs.z, Zs.w, pi.x, pi.y);
                    ffmac(fb[u][2], fb[u][3], Zs.z, Zs.w, pr.x, pr.y);
                    ffmac(fb[u][2], fb[u][3], -Zs.x, -Zs.y, pi.x, pi.y);
                  }
                }
              }
            }
          } else
#pragma unroll
          for (int u = 0; u < kQP; ++u) {
            const int q = q0 + u;
            if (q < Qn) {
              const int n = H.lev[q], s = H.stride[q], co = H.coff[q];
              const int nk = (kd >> (H.db * q)) & H.dm, nl = (ld >> (H.db * q)) & H.dm;
              const double c1 = S.cu[co + nk], c2 = S.cd[co + nl], c3 = S.cd[co + nk], c4 = S.cu[co + nl];
              const double2 x1 = nb(nk + 1 < n ? s : 0, 0);
              const double2 x2 = nb(0, nl > 0 ? -s : 0);
              const double2 x3 = nb(nk > 0 ? -s : 0, 0);
              const double2 x4 = nb(0, nl + 1 < n ? s : 0);
              const double pr = fma(-c2, x2.x, c1 * x1.x);
              const double pi = fma(-c2, x2.y, c1 * x1.y);
              const double rr = fma(-c4, x4.x, c3 * x3.x);
              const double ri = fma(-c4, x4.y, c3 * x3.y);
              if (!G.herm) {
                sar[u] = fma(Z.x, rr, fma(Z.y, ri, sar[u]));
                sai[u] = fma(Z.y, rr, fma(-Z.x, ri, sai[u]));
                sdr[u] = fma(Z.x, pr, fma(Z.y, pi, sdr[u]));
                sdi[u] = fma(Z.y, pr, fma(-Z.x, pi, sdi[u]));
              } else if (g.vm >= 0) {
                // Hermitian Z and zhat, A = Z conj(R), B = Z conj(P): the element
                // and its mirror (l, k) add A - conj(B) to the g_a sum and
                // B - conj(A), its negated conjugate, to the g_ad sum
                const double dr = rr - pr, di = ri - pi, ur = rr + pr, ui = ri + pi;
                sar[u] = fma(Z.x, dr, fma(Z.y, di, sar[u]));
                sai[u] = fma(Z.y, ur, fma(-Z.x, ui, sai[u]));
              } else {
                // a diagonal element of Hermitian Z and zhat has conj(R) = -P, so
                // B = -conj(A): it adds A to g_a and its negated conjugate to g_ad
                sar[u] = fma(Z.x, rr, fma(Z.y, ri, sar[u]));
                sai[u] = fma(Z.y, rr, fma(-Z.x, ri, sai[u]));
              }
            }
          }
          if (last) {
            // qhat^j = 2 zhat - qhat^{j+1}: no other thread reads this element in the pass
            const double2 zz = zh[o], ll = P.lam[o];
            double2 ln = make_double2(fma(2.0, zz.x, -ll.x), fma(2.0, zz.y, -ll.y));
            if (penal) {
              // the running penalty's source gamma1 beta_i/M dt beta(t_j) g(q^j) (Appendix B)
              const double2 qn = P.qb[o], t = P.tar[(size_t)b * V + v];
              const double2 qj = make_double2(fma(2.0, Z.x, -qn.x), fma(2.0, Z.y, -qn.y));
              P.qb[o] = qj;
              const double pw = H.gamma1 * P.wgt[b] * P.pen[j];
              if (H.kind == LB_J_FROB) {
                ln.x = fma(pw, qj.x - t.x, ln.x);
                ln.y = fma(pw, qj.y - t.y, ln.y);
              } else {
                const double ls = pw * linear_sign(H.kind);
                ln.x = fma(ls, t.x, ln.x);
                ln.y = fma(ls, t.y, ln.y);
              }
            }
            P.lam[o] = ln;
            if (apred) grid_commit<true>(P, ahist, o, (size_t)G.M * G.Vh, v);
          }
        }
        if constexpr (FF) {
#pragma unroll
          for (int u = 0; u < kQP; ++u) {
            sar[u] = f32_to_f64(fa[u][0]) + f32_to_f64(fa[u][1]);
            sai[u] = f32_to_f64(fa[u][2]) + f32_to_f64(fa[u][3]);
            sdr[u] = f32_to_f64(fb[u][0]) + f32_to_f64(fb[u][1]);
            sdi[u] = f32_to_f64(fb[u][2]) + f32_to_f64(fb[u][3]);
          }
        }
        if (G.herm) {
          // the g_ad sum of Hermitian Z and zhat is minus the conjugate of the g_a sum
#pragma unroll
          for (int u = 0; u < kQP; ++u) {
            sdr[u] = -sar[u];
            sdi[u] = sai[u];
          }
        }
#pragma unroll
        for (int u = 0; u < kQP; ++u) {
          const int q = q0 + u;
          if (q < Qn) {
            const double r = warp_sum4(sar[u], sai[u], sdr[u], sdi[u], lane);
            if ((lane & 7) == 0) S.red[(lane >> 3) * 8 + warp] = r;
            __syncthreads();
            if (threadIdx.x < 4) {
              double t = 0.0;
              for (int w = 0; w < nwarps; ++w) t += S.red[threadIdx.x * 8 + w];
              P.partials[((size_t)blockIdx.x * LB_MAXQ + q) * 4 + threadIdx.x] = t;
            }
            __syncthreads();
          }
        }
      }
      if (apred) {
        ahist.advance();
        if (ahist.m >= kAnchorSteps) ahist.m = 0;
      }
      if (!grid_sync(P.bar, gridDim.x, P.spin_limit > 0 ? P.spin_limit : kSpinLimit)) {
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
    atomicAdd(&P.status->diters[1], dit_rec);
    atomicAdd(&P.status->diters[2], dit_adj);
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
    P.J[i] = merit_value(P.kind, t) + (P.gamma1 != 0.0 ? P.gamma1 * P.jpen[i] : 0.0);
  }
}
}  // namespace

// ---------------------------------------------------------------------------
// launchers

size_t grid_smem_bytes(int ncoef, int njcoef) { return grid_smem_bytes_impl(ncoef, njcoef); }

int grid_blocks(int backward, int ff, size_t smem) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  const void* k = backward ? (ff ? (const void*)k_backward_grid<true> : (const void*)k_backward_grid<false>)
                           : (ff ? (const void*)k_sweep_grid<true> : (const void*)k_sweep_grid<false>);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kGridThreads, smem) != cudaSuccess) return 0;
  const int n = nsm * per;
  return n < kMaxGridBlocks ? n : kMaxGridBlocks;
}

cudaError_t launch_sweep_grid(const ProbDev* d_prob, int mode, int init_from_q0, int tape, int64_t j0, int64_t j1,
                              double2* x, int nstates, int nblocks, size_t smem, int ff, cudaStream_t s) {
  int m = mode, in = init_from_q0, tp = tape, a = (int)j0, b = (int)j1, ns = nstates;
  const ProbDev* p = d_prob;
  double2* xx = x;
  void* args[] = {(void*)&p, (void*)&m, (void*)&in, (void*)&tp, (void*)&a, (void*)&b, (void*)&xx, (void*)&ns};
  const void* k = ff ? (const void*)k_sweep_grid<true> : (const void*)k_sweep_grid<false>;
  return cudaLaunchCooperativeKernel(k, dim3(nblocks), dim3(kGridThreads), args, smem, s);
}

cudaError_t launch_backward_grid(const ProbDev* d_prob, int nblocks, size_t smem, int ff, cudaStream_t s) {
  const ProbDev* p = d_prob;
  void* args[] = {(void*)&p};
  const void* k = ff ? (const void*)k_backward_grid<true> : (const void*)k_backward_grid<false>;
  return cudaLaunchCooperativeKernel(k, dim3(nblocks), dim3(kGridThreads), args, smem, s);
}

cudaError_t launch_objective_states(const ProbDev* d_prob, int M, cudaStream_t s) {
  k_objective_states<<<M, 256, 0, s>>>(d_prob);
  return cudaGetLastError();
}

}  // namespace lbk
