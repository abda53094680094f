// Host side of the C ABI declared in include/lindblad_gb300.h.
//
// The library never allocates device memory: a system computes its workspace
// size, the caller binds device memory, and every table, state and result
// lives in that workspace.  Kernels are launched on the caller's stream.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lb_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call, where)                          \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// One region of the workspace.
struct Region {
  size_t off = 0, bytes = 0;
};

struct Layout {
  Region prob, status, items, sysp, cu, cd, jf, ja, digits, D, Dinv, alpha, carriers, ctab, q0, tar, wgt, qT, ckpt, seg,
      gproj, gsum, sfac, pen, qb, jpen, mpart, pmap, Ginv, hgp, hgm, fgp, fgm, dfA, dfB, Dinvf, zsA, zsB, J, G, grad, gateV, emap, efull, zA, zB, lam, qf, partials, gslots, bar, hist, histf,
      hkl;
  size_t total = 0;
};

}  // namespace

struct lb_system {
  // description (Sec. II), frequencies in rad/ns, rates in 1/ns
  int Q = 0;
  int levels[LB_MAXQ] = {};
  int essential[LB_MAXQ] = {};
  double det[LB_MAXQ] = {}, kerr[LB_MAXQ] = {}, g1[LB_MAXQ] = {}, g2[LB_MAXQ] = {};
  double xkerr[LB_MAXQ * LB_MAXQ] = {};
  double T = 0.0, h = 0.0;
  int64_t NT = 0;
  int N = 0, V = 0, Ne = 0;
  // controls (eq. rotctrl)
  bool ctrl_defined = false;
  int Ns = 0;
  double Tc = 0.0;  // horizon the B-splines span; 0 = the final time T
  int nf[LB_MAXQ] = {};
  std::vector<double> carriers;  // rad/ns
  std::vector<double> alpha;     // GHz, [q][f][s][re, im]
  int n_params = 0;
  // states and objective (Sec. III).  Of two states that are each other's
  // conjugate transpose, with targets that are too, only the first is
  // integrated (Lindblad's equation and the implicit midpoint step commute
  // with the conjugate transpose, so the second's final state, merit and
  // gradient share follow from the first's); M counts the integrated states.
  int M = 0;
  int Mu = 0;                  // states given by lb_states_set
  int pairing = 1;             // integrate one state of each conjugate pair (lb_set_pairing)
  std::vector<int32_t> pmap;   // [Mu] integrated index * 2 (+1 when the state is its conjugate transpose)
  std::vector<int32_t> evo;    // [M] lb_states_set index of each integrated state
  std::vector<double> rho0;    // [Mu] kept only while no workspace is bound
  std::vector<double> wgt_u;   // [Mu] beta_u / Mu
  std::vector<double> wgt;     // [M] sum of beta_u / Mu over the states each one stands for
  int kind = LB_J_FROB;
  int target_mode = 0;  // 0 none, 1 explicit, 2 gate
  std::vector<double> targets;
  std::vector<double> gateV;
  double gamma2 = 0.0;
  // solver
  int method = LB_SOLVER_JACOBI;
  int krylov = 0;  // GMRES cycle length that fits shared memory (decided at bind)
  int dbits = 4;   // bits per packed digit of a basis index
  // Jaynes-Cummings pairs p < q with g != 0: g and eta = omega_p^rot - omega_q^rot (rad/ns)
  std::vector<int> jp, jq;
  std::vector<double> jg, je;
  double rtol = 1e-15;
  int max_iter = 200;
  int K = 100;       // requested checkpoint interval; < 0 = automatic (effective_K)
  int sweep = LB_SWEEP_AUTO;
  int symmetry = LB_SYM_AUTO;
  int pred = LB_PRED_AUTO;  // restart period of the forward predictor as requested (lb_set_predictor)
  int pred_order = lbk::kDefaultRingOrder;  // its order (grid and one-CTA sweeps)
  long long spin_limit = 0;  // polls of a grid-barrier wait (0: the kernels' default; lb_set_wait_limit)
  int diffit = 1;            // single-precision difference iterations in the grid sweeps (lb_set_difference_iterations)
  int precision = LB_PREC_F64;  // arithmetic of the grid sweeps' FP64 iterations (lb_set_precision)
  double gamma1 = 0.0, pen_a = 1.0;  // running penalty (one CTA per state)
  bool rho_herm = false;  // every initial state exactly Hermitian
  bool tar_herm = false;  // every explicit target exactly Hermitian (gate targets: always)
  bool rho_finite = true;  // no NaN or Inf in the initial states
  int gblocks = 0;   // cooperative grid size of the forward grid sweep
  int gblocks_b = 0;  // ... and of the backward one
  size_t gsmem = 0;  // its dynamic shared memory
  bool cluster = false;      // cluster-split sweeps (decided at bind)
  bool tapes_packed = false;  // the bound workspace holds the grid sweeps' tapes packed (k <= l)
  lbk::ClusterConfig cc{};
  // device binding
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t bind_stream = nullptr;
  cudaEvent_t upload_done = nullptr;
  Layout L;
  ProbDev hp{};
  ProbDev* dp = nullptr;
  WorkItem* d_items = nullptr;
  lbk::ResidentConfig rc{};
  bool ctab_dirty = true;
  lb_stats last{};
  int launches = 0;
  bool timing = false;
  bool timed_fwd = false, timed_bwd = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // forward start/end, backward start/end
};

struct lb_batch {
  std::vector<lb_system*> sys;
  std::vector<int64_t> grad_off;
  int64_t n_grad = 0;
  int n_items = 0;
  int max_param_warps = 0;
  lbk::ResidentConfig rc{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  ProbDev* d_probs = nullptr;
  WorkItem* d_items = nullptr;
  int64_t* d_grad_off = nullptr;
  double* d_G = nullptr;
  double* d_grad = nullptr;
  DevStatus* d_st = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  lb_stats last{};
};

namespace {

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Grid-wide sweeps for states that do not fit one CTA's shared memory, or
// when asked for; AUTO also prefers them when few states leave most SMs idle.
bool use_grid(const lb_system* s) {
  if (s->V > lbk::kMaxResidentV) return true;
  if (s->method == LB_SOLVER_GMRES) return false;  // GMRES runs one CTA per state
  if (s->gamma1 != 0.0) return s->sweep == LB_SWEEP_GRID;  // the running penalty: AUTO keeps small states per CTA
  if (s->sweep == LB_SWEEP_GRID) return true;
  if (s->sweep == LB_SWEEP_RESIDENT || s->sweep == LB_SWEEP_CLUSTER) return false;
  return s->V >= 1024 && s->M < 64;
}

int n_coef(const lb_system* s) {
  int n = 0;
  for (int q = 0; q < s->Q; ++q) n += s->levels[q];
  return n;
}
int n_jcoef(const lb_system* s) {
  int n = 0;
  for (int q = 0; q < s->Q; ++q) n += s->levels[q] * s->levels[q];
  return n;
}
int n_carriers_total(const lb_system* s) {
  int n = 0;
  for (int q = 0; q < s->Q; ++q) n += s->nf[q];
  return n;
}

// Checkpoint interval actually used: the requested one, or for an automatic
// request the full stage tape (0) when it takes at most kTapeBudget bytes,
// else checkpoints every 100 steps.
constexpr size_t kTapeBudget = size_t(8) << 30;
int effective_K(const lb_system* s) {
  if (s->K >= 0) return s->K;
  const size_t tape = sizeof(double2) * (size_t)s->M * (size_t)s->NT * (size_t)s->V;
  if (tape <= kTapeBudget) return 0;
  return s->NT < 100 ? (int)s->NT : 100;
}

// Restart period of the forward first-iterate predictor in effect:
// LB_PRED_NONE (no forward predictor), 0 (never restarts, full stage tape
// only) or R > 0 (restarts at every step j with j % R == 0; R divides K
// with checkpoints, so that every checkpoint is a restart point).
int effective_pred(const lb_system* s) {
  if (s->method == LB_SOLVER_NEUMANN || s->pred == LB_PRED_NONE) return LB_PRED_NONE;
  const int K = effective_K(s);
  if (s->pred == LB_PRED_AUTO) return K;
  return s->pred;
}

// The grid sweep's running penalty sums each step's merit per block over the
// at most 4 states a block's contiguous chunk of elements covers: check that
// for both element counts per state (all N^2, or N (N + 1) / 2 under the
// Hermitian symmetry, which is decided per call).
bool grid_chunks_cover_few_states(const lb_system* s) {
  const long long vh[2] = {(long long)s->V, (long long)s->N * (s->N + 1) / 2};
  for (long long Vh : vh) {
    const long long total = (long long)s->M * Vh;
    const long long per = (total + s->gblocks - 1) / s->gblocks;
    const long long chunk = (per + 31) / 32 * 32;
    for (long long e0 = 0; e0 < total; e0 += chunk) {
      const long long e1 = std::min(total, e0 + chunk);
      if ((e1 - 1) / Vh - e0 / Vh + 1 > 4) return false;
    }
  }
  return true;
}

// every checkpoint must be a restart point of the forward predictor
int check_predictor(const lb_system* s) {
  const int K = effective_K(s), R = effective_pred(s);
  if (K > 0 && R == 0) return fail(LB_EINVAL, "a predictor that never restarts needs the full stage tape (K = 0)");
  if (K > 0 && R > 0 && K % R != 0)
    return fail(LB_EINVAL, "the predictor's restart period must divide the checkpoint interval");
  return LB_OK;
}

// the recompute needs its own predictor history when it predicts
bool recompute_predicts(const lb_system* s) { return effective_K(s) > 0 && effective_pred(s) > 0; }

// Cluster sweep configuration of this system with 2 or 4 lanes per half
// pair (cs = false / true; a subsystem's control terms, or a Jaynes-Cummings
// pair, make one half pair); C == 0 when it cannot apply.
lbk::ClusterConfig cluster_cfg(const lb_system* s, bool cs) {
  if (use_grid(s) || s->sweep == LB_SWEEP_RESIDENT || s->method == LB_SOLVER_GMRES) return lbk::ClusterConfig{};
  lbk::ClusterConfig cc = lbk::cluster_config(s->V, s->Q + (int)s->jp.size(), n_coef(s), n_jcoef(s), s->N, cs);
  cc.pen = s->gamma1 != 0.0;
  return cc;
}

// complex values of the GMRES Krylov basis in shared memory (0 for the
// fixed-point solvers)
size_t kry_elems(const lb_system* s) {
  return s->method == LB_SOLVER_GMRES ? (size_t)(s->krylov + 1) * s->V : 0;
}

// GMRES cycle length for this system on the current device; with GMRES
// chosen, check that it can run (one CTA per state, basis in shared memory).
int decide_krylov(lb_system* s) {
  int dev = 0, optin = 0;
  LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  LB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute");
  s->krylov = s->V <= lbk::kMaxResidentV ? lbk::gmres_krylov_dim(s->V, n_coef(s), n_jcoef(s), s->N, (size_t)optin) : 0;
  if (s->method != LB_SOLVER_GMRES) return LB_OK;
  if (s->sweep == LB_SWEEP_GRID || s->sweep == LB_SWEEP_CLUSTER)
    return fail(LB_EINVAL, "GMRES runs in the one-CTA-per-state sweep only (LB_SWEEP_RESIDENT or AUTO)");
  if (s->krylov <= 0)
    return fail(LB_EINVAL, "GMRES needs its Krylov basis in one CTA's shared memory: N^2 too large");
  s->sweep = LB_SWEEP_RESIDENT;
  return LB_OK;
}

// slots of the gradient pieces: one (summed) for grid sweeps, one per state,
// CTA and warp where cluster sweeps can run (enough for either lane layout),
// one per state otherwise
size_t gproj_slots(const lb_system* s) {
  if (use_grid(s)) return 1;
  size_t per = 1;
  for (int cs = 0; cs < 2; ++cs) {
    const lbk::ClusterConfig cc = cluster_cfg(s, cs != 0);
    if (cc.C > 0) per = std::max(per, (size_t)cc.C * (cc.threads / 32));
  }
  return (size_t)s->M * per;
}

// slots the bound sweep writes
int gproj_used(const lb_system* s) {
  if (use_grid(s)) return 1;
  return s->cluster ? s->M * s->cc.C * (s->cc.threads / 32) : s->M;
}

bool use_symmetry(const lb_system* s);
bool packed_tapes(const lb_system* s);

Layout make_layout(const lb_system* s) {
  Layout L;
  size_t off = 0;
  auto take = [&](Region& r, size_t bytes) {
    r.off = off;
    r.bytes = bytes;
    off += align_up(bytes ? bytes : 1);
  };
  const size_t V = (size_t)s->V, M = (size_t)s->M, NT = (size_t)s->NT;
  const size_t c2 = sizeof(double2);
  take(L.prob, sizeof(ProbDev));
  take(L.status, sizeof(DevStatus));
  take(L.items, sizeof(WorkItem) * M);
  take(L.sysp, sizeof(double) * (4 * s->Q + s->Q * s->Q));
  take(L.cu, sizeof(double) * n_coef(s));
  take(L.cd, sizeof(double) * n_coef(s));
  take(L.jf, sizeof(double) * n_jcoef(s));
  take(L.ja, sizeof(double) * n_jcoef(s));
  take(L.digits, sizeof(uint32_t) * s->N);
  take(L.D, c2 * V);
  take(L.Dinv, c2 * V);
  take(L.alpha, sizeof(double) * s->n_params);
  take(L.carriers, sizeof(double) * n_carriers_total(s));
  take(L.ctab, c2 * NT * (s->Q + s->jp.size()));
  take(L.sfac, sizeof(double) * NT);
  take(L.pen, sizeof(double) * NT);
  take(L.qb, s->gamma1 != 0.0 ? c2 * M * V : 0);
  take(L.jpen, s->gamma1 != 0.0 ? sizeof(double) * M : 0);
  take(L.mpart, s->gamma1 != 0.0 && use_grid(s) ? sizeof(double) * lbk::kMaxGridBlocks * 4 : 0);
  take(L.q0, c2 * M * V);
  take(L.tar, c2 * M * V);
  take(L.wgt, sizeof(double) * M);
  take(L.qT, c2 * M * V);
  const int K = effective_K(s);
  const size_t nck = K > 0 ? (NT + K - 1) / K : NT;
  const size_t Vt = packed_tapes(s) ? (size_t)s->N * (s->N + 1) / 2 : V;  // entries per state in the tapes
  take(L.ckpt, c2 * M * nck * Vt);
  take(L.seg, K > 0 ? c2 * M * (size_t)K * Vt : 0);
  const bool grid = use_grid(s);
  take(L.gproj, c2 * gproj_slots(s) * NT * s->Q * 2);
  take(L.gsum, c2 * NT * s->Q * 2);
  take(L.J, sizeof(double) * M);
  take(L.G, sizeof(double));
  take(L.grad, sizeof(double) * s->n_params);
  const size_t Ne = (size_t)s->Ne;
  take(L.gateV, s->target_mode == 2 ? c2 * Ne * Ne : 0);
  take(L.emap, s->target_mode == 2 ? sizeof(int32_t) * s->N : 0);
  take(L.efull, s->target_mode == 2 ? sizeof(int32_t) * Ne : 0);
  take(L.zA, grid ? c2 * M * V : 0);
  take(L.zB, grid ? c2 * M * V : 0);
  take(L.lam, grid ? c2 * M * V : 0);
  take(L.qf, grid ? c2 * M * V : 0);
  take(L.partials, grid ? sizeof(double) * lbk::kMaxGridBlocks * LB_MAXQ * 4 : 0);
  take(L.gslots, grid ? sizeof(unsigned long long) * 5 * M : 0);
  take(L.bar, grid ? sizeof(GridBar) : 0);
  take(L.hist, c2 * lbk::kRingOrder * M * V);
  take(L.histf, recompute_predicts(s) ? c2 * lbk::kRingOrder * M * V : 0);
  // the powers g^m, g^-m of each predictor ring's anchor frame, and 1/g
  take(L.Ginv, c2 * V);
  take(L.hgp, c2 * M * V);
  take(L.hgm, c2 * M * V);
  take(L.fgp, recompute_predicts(s) ? c2 * M * V : 0);
  take(L.fgm, recompute_predicts(s) ? c2 * M * V : 0);
  take(L.dfA, grid ? sizeof(float2) * M * V : 0);
  take(L.dfB, grid ? sizeof(float2) * M * V : 0);
  take(L.Dinvf, grid ? sizeof(float2) * V : 0);
  take(L.zsA, grid && s->precision == LB_PREC_F32X2 ? sizeof(float4) * M * V : 0);
  take(L.zsB, grid && s->precision == LB_PREC_F32X2 ? sizeof(float4) * M * V : 0);
  take(L.hkl, sizeof(uint32_t) * (size_t)s->N * (s->N + 1) / 2);
  take(L.pmap, sizeof(int32_t) * (size_t)s->Mu);
  L.total = off;
  return L;
}

template <class T>
T* at(const lb_system* s, const Region& r) {
  return reinterpret_cast<T*>(s->ws + r.off);
}

int check_ready(const lb_system* s, bool need_bound) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (!s->ctrl_defined) return fail(LB_EINVAL, "controls not defined (lb_controls_define)");
  if (s->M <= 0) return fail(LB_EINVAL, "no initial states (lb_states_set)");
  if (need_bound && !s->ws) return fail(LB_EINVAL, "no workspace bound (lb_bind_workspace)");
  if (need_bound && s->tapes_packed && !use_symmetry(s)) {
    // a NaN or Inf in a state also breaks the symmetry test: report it as the
    // sweeps would (at the first step)
    if (!s->rho_finite) return fail(LB_ENAN, "an initial state holds NaN or Inf (time step 0)");
    return fail(LB_EINVAL,
                "the workspace was bound for Hermitian states and targets (packed tapes); bind a new one for these");
  }
  return LB_OK;
}

// Make `stream` wait for the uploads issued on the bind stream.
int order_after_uploads(lb_system* s, cudaStream_t stream) {
  if (stream == s->bind_stream) return LB_OK;
  LB_CUDA(cudaEventRecord(s->upload_done, s->bind_stream), "cudaEventRecord");
  LB_CUDA(cudaStreamWaitEvent(stream, s->upload_done, 0), "cudaStreamWaitEvent");
  return LB_OK;
}

// the elements k <= l, column by column, as k | l << 16 (N <= 2^15): the
// element order of the grid sweeps under the Hermitian symmetry.
// The pageable source is staged before cudaMemcpyAsync returns.
int upload_symmetry_map(lb_system* s, cudaStream_t st) {
  std::vector<uint32_t> hkl;
  hkl.reserve((size_t)s->N * (s->N + 1) / 2);
  for (int l = 0; l < s->N; ++l)
    for (int k = 0; k <= l; ++k) hkl.push_back((uint32_t)k | ((uint32_t)l << 16));
  LB_CUDA(cudaMemcpyAsync(at<uint32_t>(s, s->L.hkl), hkl.data(), sizeof(uint32_t) * hkl.size(),
                          cudaMemcpyHostToDevice, st),
          "upload symmetry map");
  return LB_OK;
}

// b == a^+ entry by entry (column-major N x N complex, interleaved)
bool is_conj_transpose(const double* a, const double* b, int N) {
  for (int l = 0; l < N; ++l)
    for (int k = 0; k < N; ++k) {
      const size_t p = (size_t)2 * (k + (size_t)N * l), q = (size_t)2 * (l + (size_t)N * k);
      if (b[p] != a[q] || b[p + 1] != -a[q + 1]) return false;
    }
  return true;
}

// Conjugate pairs among the Mu states `rho` (with explicit targets `tar`, or
// null when the targets follow from the states or are all the same real
// diagonal): state w after u with rho_w = rho_u^+ (and tar_w = tar_u^+) is
// carried by u.  pmap[u] = 2 e (+1 for a carried state), evo[e] = u.
void find_pairs(const lb_system* s, const double* rho, const double* tar, std::vector<int32_t>& pmap,
                std::vector<int32_t>& evo) {
  const int Mu = s->Mu, N = s->N;
  const size_t st = (size_t)2 * s->V;
  pmap.assign(Mu, -1);
  evo.clear();
  for (int u = 0; u < Mu; ++u) {
    if (pmap[u] >= 0) continue;
    const int e = (int)evo.size();
    evo.push_back(u);
    pmap[u] = 2 * e;
    if (!s->pairing) continue;
    for (int w = u + 1; w < Mu; ++w) {
      if (pmap[w] >= 0) continue;
      if (!is_conj_transpose(rho + u * st, rho + w * st, N)) continue;
      if (tar && !is_conj_transpose(tar + u * st, tar + w * st, N)) continue;
      pmap[w] = 2 * e + 1;
      break;
    }
  }
}

// explicit targets that must pair with the states (null: none, or every
// state's target the same real diagonal N_m)
const double* pairing_targets(const lb_system* s) {
  return (s->target_mode == 1 && s->kind != LB_J_NM && !s->targets.empty()) ? s->targets.data() : nullptr;
}

// the integrated states' weights from the per-state ones
void apply_pairs(lb_system* s) {
  s->M = (int)s->evo.size();
  s->wgt.assign(s->M, 0.0);
  for (int u = 0; u < s->Mu; ++u) s->wgt[s->pmap[u] >> 1] += s->wgt_u[u];
}

// re-decide the pairs from the host copies (no workspace bound)
void update_pairs(lb_system* s) {
  if (s->Mu < 1 || s->rho0.empty()) return;
  find_pairs(s, s->rho0.data(), pairing_targets(s), s->pmap, s->evo);
  apply_pairs(s);
}

// with a workspace bound the pairs are fixed: new states or targets must pair
// the same way
int check_pairs(lb_system* s, const double* rho, const double* tar) {
  std::vector<int32_t> pm, ev;
  find_pairs(s, rho, tar, pm, ev);
  if (pm != s->pmap)
    return fail(LB_EINVAL, "the states' conjugate pairs differ from those the workspace was bound with (rebind)");
  return LB_OK;
}

// the integrated states of the Mu given ones (pageable; staged before cudaMemcpyAsync returns)
std::vector<double> gather_states(const lb_system* s, const double* a) {
  const size_t st = (size_t)2 * s->V;
  std::vector<double> out(st * s->M);
  for (int e = 0; e < s->M; ++e) std::memcpy(out.data() + e * st, a + s->evo[e] * st, sizeof(double) * st);
  return out;
}

int upload_states(lb_system* s, const double* rho0, cudaStream_t st) {
  const size_t bytes = sizeof(double2) * (size_t)s->M * s->V;
  if (s->M == s->Mu) {
    LB_CUDA(cudaMemcpyAsync(at<double2>(s, s->L.q0), rho0, bytes, cudaMemcpyHostToDevice, st), "upload states");
  } else {
    const std::vector<double> g = gather_states(s, rho0);
    LB_CUDA(cudaMemcpyAsync(at<double2>(s, s->L.q0), g.data(), bytes, cudaMemcpyHostToDevice, st), "upload states");
  }
  LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.wgt), s->wgt.data(), sizeof(double) * s->M, cudaMemcpyHostToDevice, st),
          "upload weights");
  return LB_OK;
}

int upload_targets(lb_system* s, cudaStream_t st) {
  const size_t bytes = sizeof(double2) * (size_t)s->M * s->V;
  if (s->target_mode == 1) {
    if (s->M == s->Mu) {
      LB_CUDA(cudaMemcpyAsync(at<double2>(s, s->L.tar), s->targets.data(), bytes, cudaMemcpyHostToDevice, st),
              "upload targets");
    } else {
      const std::vector<double> g = gather_states(s, s->targets.data());
      LB_CUDA(cudaMemcpyAsync(at<double2>(s, s->L.tar), g.data(), bytes, cudaMemcpyHostToDevice, st),
              "upload targets");
    }
  } else if (s->target_mode == 2) {
    // essential <-> full index maps (subsystem 0 most significant)
    std::vector<int32_t> emap(s->N, -1), efull(s->Ne, 0);
    for (int a = 0; a < s->Ne; ++a) {
      int rem = a, k = 0, mul = 1;
      for (int q = s->Q - 1; q >= 0; --q) {
        const int dg = rem % s->essential[q];
        rem /= s->essential[q];
        k += dg * mul;
        mul *= s->levels[q];
      }
      efull[a] = k;
      emap[k] = a;
    }
    LB_CUDA(cudaMemcpyAsync(at<int32_t>(s, s->L.emap), emap.data(), sizeof(int32_t) * s->N, cudaMemcpyHostToDevice, st),
            "upload gate map");
    LB_CUDA(cudaMemcpyAsync(at<int32_t>(s, s->L.efull), efull.data(), sizeof(int32_t) * s->Ne, cudaMemcpyHostToDevice,
                            st),
            "upload gate map");
    LB_CUDA(cudaMemcpyAsync(at<double2>(s, s->L.gateV), s->gateV.data(), sizeof(double2) * s->Ne * s->Ne,
                            cudaMemcpyHostToDevice, st),
            "upload gate");
    // pageable sources above are staged before cudaMemcpyAsync returns
    LB_CUDA(lbk::launch_gate_targets(s->hp, at<double2>(s, s->L.gateV), at<int32_t>(s, s->L.emap),
                                     at<int32_t>(s, s->L.efull), s->Ne, st),
            "gate targets kernel");
  } else {
    LB_CUDA(cudaMemsetAsync(at<double2>(s, s->L.tar), 0, bytes, st), "clear targets");
  }
  return LB_OK;
}

// every M x N x N complex matrix (column-major, interleaved) Hermitian to
// rounding: each entry within 64 eps max|entry| of the conjugate of its
// transposed entry (an outer product psi psi^+ formed with fused multiply-adds
// is Hermitian only to that level)
bool hermitian_matrices(const double* a, int M, int N) {
  const size_t NN = (size_t)N * N;
  for (int i = 0; i < M; ++i) {
    const double* m = a + 2 * (size_t)i * NN;
    double amax = 0.0;
    for (size_t t = 0; t < 2 * NN; ++t) amax = std::max(amax, std::fabs(m[t]));
    const double tol = 64.0 * 2.220446049250313e-16 * amax;
    for (int l = 0; l < N; ++l)
      for (int k = 0; k <= l; ++k) {
        const size_t p = (size_t)2 * (k + (size_t)N * l), q = (size_t)2 * (l + (size_t)N * k);
        if (!(std::fabs(m[p] - m[q]) <= tol) || !(std::fabs(m[p + 1] + m[q + 1]) <= tol)) return false;
      }
  }
  return true;
}

// the Hermitian symmetry runs in every sweep kind: grid, one CTA per state
// (fixed points and GMRES) and, when asked for explicitly, cluster (LB_SYM_AUTO
// leaves it out there: the cluster sweep's steps are bound by latency, not by
// the number of elements, and the pushes to the mirrors made the three-state
// gate workload 5 % slower)
bool use_symmetry(const lb_system* s) {
  if (s->symmetry == LB_SYM_NONE || !s->rho_herm || !(s->target_mode == 2 || s->tar_herm)) return false;
  if (s->symmetry == LB_SYM_HERMITIAN || use_grid(s)) return true;
  return !s->cluster;
}

// The grid sweeps keep the checkpoint and segment tapes packed (the k <= l
// entries of each state) under the Hermitian symmetry, so a workspace bound
// while the states and targets are Hermitian sizes them N (N + 1) / 2 per
// state instead of N^2.
bool packed_tapes(const lb_system* s) { return use_grid(s) && use_symmetry(s); }

// re-upload the problem block when the symmetry decision changed (bound systems)
int refresh_symmetry(lb_system* s) {
  if (!s->ws) return LB_OK;
  const int h = use_symmetry(s) ? 1 : 0;
  if (h == s->hp.herm) return LB_OK;
  s->hp.herm = h;
  LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, s->bind_stream), "upload problem");
  return LB_OK;
}

// NVTX range over a host scope (the enqueueing of a sweep; visible in
// Nsight timelines beside the kernels it launches)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int upload_controls(lb_system* s, cudaStream_t st) {
  if (s->n_params)
    LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.alpha), s->alpha.data(), sizeof(double) * s->n_params,
                            cudaMemcpyHostToDevice, st),
            "upload alpha");
  s->ctab_dirty = true;
  return LB_OK;
}

void fill_prob(lb_system* s) {
  ProbDev& P = s->hp;
  std::memset(&P, 0, sizeof(P));
  P.Q = s->Q;
  P.N = s->N;
  P.M = s->M;
  P.NT = (int32_t)s->NT;
  P.V = s->V;
  P.K = effective_K(s);
  P.n_ckpt = P.K > 0 ? (int32_t)((s->NT + P.K - 1) / P.K) : (int32_t)s->NT;
  P.max_iter = s->max_iter;
  P.method = s->method;
  P.krylov = s->krylov;
  P.dbits = s->dbits;
  P.npair = (int32_t)s->jp.size();
  P.cq = s->Q + P.npair;
  for (int k = 0; k < P.npair; ++k) {
    P.jp[k] = s->jp[k];
    P.jq[k] = s->jq[k];
    P.jg[k] = s->jg[k];
    P.je[k] = s->je[k];
  }
  P.kind = s->kind;
  P.Ns = s->Ns;
  P.n_params = s->n_params;
  P.h = s->h;
  P.rtol = s->rtol;
  P.T = s->T;
  P.Tc = s->Tc > 0.0 ? s->Tc : s->T;
  P.gamma2 = s->gamma2;
  int stride = 1, co = 0, jo = 0, fo = 0, ao = 0;
  for (int q = s->Q - 1; q >= 0; --q) {
    P.stride[q] = stride;
    stride *= s->levels[q];
  }
  for (int q = 0; q < s->Q; ++q) {
    P.levels[q] = s->levels[q];
    P.coff[q] = co;
    co += s->levels[q];
    P.joff[q] = jo;
    jo += s->levels[q] * s->levels[q];
    P.nf[q] = s->nf[q];
    P.foff[q] = fo;
    fo += s->nf[q];
    P.aoff[q] = ao;
    ao += 2 * s->Ns * s->nf[q];
    P.jump[q] = 0.5 * s->h * s->g1[q];
  }
  P.ncoef = co;
  P.njcoef = jo;
  P.sysp = at<double>(s, s->L.sysp);
  P.cu = at<double>(s, s->L.cu);
  P.cd = at<double>(s, s->L.cd);
  P.jf = at<double>(s, s->L.jf);
  P.ja = at<double>(s, s->L.ja);
  P.digits = at<uint32_t>(s, s->L.digits);
  P.D = at<double2>(s, s->L.D);
  P.Dinv = at<double2>(s, s->L.Dinv);
  P.alpha = at<double>(s, s->L.alpha);
  P.carriers = at<double>(s, s->L.carriers);
  P.ctab = at<double2>(s, s->L.ctab);
  P.q0 = at<double2>(s, s->L.q0);
  P.tar = at<double2>(s, s->L.tar);
  P.wgt = at<double>(s, s->L.wgt);
  P.qT = at<double2>(s, s->L.qT);
  P.ckpt = at<double2>(s, s->L.ckpt);
  P.seg = at<double2>(s, s->L.seg);
  P.gproj = at<double2>(s, s->L.gproj);
  P.gsum = at<double2>(s, s->L.gsum);
  P.sfac = at<double>(s, s->L.sfac);
  P.pen = at<double>(s, s->L.pen);
  P.qb = at<double2>(s, s->L.qb);
  P.jpen = at<double>(s, s->L.jpen);
  P.mpart = at<double>(s, s->L.mpart);
  P.gamma1 = s->gamma1;
  P.pen_a = s->pen_a;
  P.J = at<double>(s, s->L.J);
  P.G = at<double>(s, s->L.G);
  P.grad = at<double>(s, s->L.grad);
  P.status = at<DevStatus>(s, s->L.status);
  const bool grid = use_grid(s);
  P.gM = gproj_used(s);
  P.grid_blocks = grid ? std::max(s->gblocks, s->gblocks_b) : 0;
  if (grid) {
    P.zA = at<double2>(s, s->L.zA);
    P.zB = at<double2>(s, s->L.zB);
    P.lam = at<double2>(s, s->L.lam);
    P.qf = at<double2>(s, s->L.qf);
    P.partials = at<double>(s, s->L.partials);
    P.gslots = at<unsigned long long>(s, s->L.gslots);
    P.bar = at<GridBar>(s, s->L.bar);
  }
  P.hkl = at<uint32_t>(s, s->L.hkl);
  P.herm = use_symmetry(s) ? 1 : 0;
  P.hist = at<double2>(s, s->L.hist);
  P.histf = at<double2>(s, s->L.histf);
  P.Ginv = at<double2>(s, s->L.Ginv);
  P.hgp = at<double2>(s, s->L.hgp);
  P.hgm = at<double2>(s, s->L.hgm);
  P.fgp = at<double2>(s, s->L.fgp);
  P.fgm = at<double2>(s, s->L.fgm);
  P.pred_restart = effective_pred(s);
  P.pred_order = s->pred_order;
  P.spin_limit = s->spin_limit;
  P.diffit = s->diffit;
  P.dfA = grid ? at<float2>(s, s->L.dfA) : nullptr;
  P.dfB = grid ? at<float2>(s, s->L.dfB) : nullptr;
  P.Dinvf = grid ? at<float2>(s, s->L.Dinvf) : nullptr;
  // the paired-single apply covers the control and decay terms; with
  // Jaynes-Cummings pairs the iterations stay FP64
  P.ff = grid && s->precision == LB_PREC_F32X2 && s->jp.empty() ? 1 : 0;
  P.zsA = P.ff ? at<float4>(s, s->L.zsA) : nullptr;
  P.zsB = P.ff ? at<float4>(s, s->L.zsB) : nullptr;
}

int ensure_ctab(lb_system* s, cudaStream_t st) {
  if (!s->ctab_dirty) return LB_OK;
  LB_CUDA(lbk::launch_control_table(s->dp, s->hp, st), "control table kernels");
  s->launches += 2;  // control table, stopping factors
  s->ctab_dirty = false;
  return LB_OK;
}

int read_status(const DevStatus& d, lb_stats* st, int launches) {
  if (st) {
    *st = lb_stats{};
    for (int p = 0; p < 3; ++p) {
      st->phase_steps[p] = (int64_t)d.steps[p];
      st->phase_iterations[p] = (int64_t)d.iters[p];
      st->phase_diff_iterations[p] = (int64_t)d.diters[p];
      st->state_steps += (int64_t)d.steps[p];
      st->inner_iterations += (int64_t)d.iters[p];
    }
    st->max_iterations = d.max_iter_seen;
    st->kernel_launches = launches;
  }
  if (d.code == LB_ENOTCONV) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "inner solve did not converge within max_iter at time step %d", d.step);
    return fail(LB_ENOTCONV, buf);
  }
  if (d.code == LB_ENAN) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "state became NaN or Inf at time step %d", d.step);
    return fail(LB_ENAN, buf);
  }
  if (d.code == LB_ECUDA) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "a grid barrier wait gave up at time step %d", d.step);
    return fail(LB_ECUDA, buf);
  }
  return LB_OK;
}


}  // namespace

// ===========================================================================
extern "C" {

const char* lb_last_error(void) { return g_err.c_str(); }

const char* lb_version(void) { return "lindblad_gb300 0.1 (sm_103a, FP64)"; }

int lb_system_create(const lb_system_desc* d, lb_system** out) {
  if (!d || !out) return fail(LB_EINVAL, "null argument");
  if (d->Q < 1 || d->Q > LB_MAX_SUBSYSTEMS) return fail(LB_EINVAL, "Q out of range 1..8");
  if (!d->levels || !d->detuning_ghz) return fail(LB_EINVAL, "levels and detuning_ghz are required");
  if (!(d->T_ns > 0.0) || !std::isfinite(d->T_ns)) return fail(LB_EINVAL, "T_ns must be finite and > 0");
  if (d->n_steps < 1 || d->n_steps > (1LL << 30)) return fail(LB_EINVAL, "n_steps out of range");
  lb_system* s = new (std::nothrow) lb_system();
  if (!s) return fail(LB_ENOMEM, "host allocation failed");
  s->Q = d->Q;
  long long N = 1, Ne = 1;
  for (int q = 0; q < d->Q; ++q) {
    const int n = d->levels[q];
    if (n < 2 || n > LB_MAX_LEVELS) {
      delete s;
      return fail(LB_EINVAL, "levels must be in 2..64");
    }
    s->levels[q] = n;
    const int e = d->essential ? d->essential[q] : n;
    if (e < 1 || e > n) {
      delete s;
      return fail(LB_EINVAL, "essential levels must be in 1..levels");
    }
    s->essential[q] = e;
    N *= n;
    Ne *= e;
    s->det[q] = kTwoPi * d->detuning_ghz[q];
    s->kerr[q] = d->selfkerr_ghz ? kTwoPi * d->selfkerr_ghz[q] : 0.0;
    const double t1 = d->t1_us ? d->t1_us[q] : 0.0, t2 = d->t2_us ? d->t2_us[q] : 0.0;
    s->g1[q] = finite_pos(t1) ? 1.0 / (1000.0 * t1) : 0.0;
    s->g2[q] = finite_pos(t2) ? 1.0 / (1000.0 * t2) : 0.0;
    if (!std::isfinite(s->det[q]) || !std::isfinite(s->kerr[q])) {
      delete s;
      return fail(LB_EINVAL, "non-finite detuning or self-Kerr");
    }
  }
  {
    // every basis index's digits packed into 32 bits
    int nmax = 2;
    for (int q = 0; q < d->Q; ++q) nmax = std::max(nmax, s->levels[q]);
    int db = 4;
    while ((1 << db) < nmax) ++db;
    if (db * d->Q > 32) {
      delete s;
      return fail(LB_EINVAL, "Q * ceil(log2 max levels) must be <= 32");
    }
    s->dbits = db;
  }
  if (N > (1 << 15)) {
    delete s;
    return fail(LB_EINVAL, "N = prod(levels) must be <= 32768");
  }
  if (d->crosskerr_ghz)
    for (int p = 0; p < d->Q; ++p)
      for (int q = p + 1; q < d->Q; ++q) s->xkerr[p * d->Q + q] = kTwoPi * d->crosskerr_ghz[p * d->Q + q];
  s->N = (int)N;
  s->V = (int)(N * N);
  s->Ne = (int)Ne;
  s->T = d->T_ns;
  s->NT = d->n_steps;
  s->h = d->T_ns / (double)d->n_steps;
  *out = s;
  return LB_OK;
}

void lb_system_destroy(lb_system* s) {
  if (!s) return;
  if (s->upload_done) cudaEventDestroy(s->upload_done);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

static int propagate_impl(lb_system* s, cudaStream_t st, int adjoint, int64_t j0, int64_t j1, double2* x, int n_vec);

int lb_autotune(lb_system* s, void* stream, int32_t probe_steps, int32_t* choice_out) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  if (probe_steps < 1) return fail(LB_EINVAL, "probe_steps must be >= 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t steps = probe_steps < s->NT ? probe_steps : s->NT;
  struct Cand {
    int sweep, method, E;
  };
  std::vector<Cand> cands;
  // the bound workspace fixes the sweep family: grid buffers exist only for
  // grid sweeps, GMRES runs one CTA per state
  const bool grid0 = use_grid(s);
  const int methods[3] = {LB_SOLVER_JACOBI, LB_SOLVER_NEUMANN, LB_SOLVER_GMRES};
  for (int m : methods) {
    if (grid0) {
      if (m != LB_SOLVER_GMRES) cands.push_back({LB_SWEEP_GRID, m, 0});
      continue;
    }
    if (m == LB_SOLVER_GMRES && s->krylov <= 0) continue;
    for (int E = 1; E <= 8; E *= 2) {
      const int threads = ((s->V + E - 1) / E + 31) / 32 * 32;
      if (threads > 512 || (E > 1 && threads < 64)) continue;
      cands.push_back({LB_SWEEP_RESIDENT, m, E});
    }
    if (m != LB_SOLVER_GMRES && s->cc.C > 0)
      for (int cs = 0; cs < 2; ++cs)
        if (cluster_cfg(s, cs != 0).C > 0) cands.push_back({LB_SWEEP_CLUSTER, m, cs});
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LB_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
  LB_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
  const lbk::ResidentConfig rc0 = s->rc;
  const bool cl0 = s->cluster;
  const lbk::ClusterConfig cc0 = s->cc;
  const int m0 = s->method;
  float best = -1.0f;
  Cand win{-1, m0, 0};
  double2* probe = at<double2>(s, s->L.qT);
  const size_t bytes = sizeof(double2) * (size_t)s->M * s->V;
  for (const Cand& c : cands) {
    s->method = c.method;
    s->hp.method = c.method;
    s->cluster = c.sweep == LB_SWEEP_CLUSTER;
    if (s->cluster) s->cc = cluster_cfg(s, c.E != 0);
    s->hp.gM = gproj_used(s);
    s->hp.herm = use_symmetry(s) ? 1 : 0;
    if (c.sweep == LB_SWEEP_RESIDENT) {
      s->rc = lbk::resident_config(s->V, s->Q, n_coef(s), n_jcoef(s), s->N, s->jp.empty(), kry_elems(s));
      const int threads = ((s->V + c.E - 1) / c.E + 31) / 32 * 32;
      s->rc.E = c.E;
      s->rc.threads = threads;
      s->rc.QT = (c.E == 1 && s->Q <= 4 && s->jp.empty()) ? s->Q : 0;
    }
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
    LB_CUDA(cudaMemcpyAsync(probe, at<double2>(s, s->L.q0), bytes, cudaMemcpyDeviceToDevice, st), "probe states");
    // one untimed run (module loading, first-launch costs), one timed
    int r = propagate_impl(s, st, 0, 0, steps, probe, s->M);
    if (r == LB_OK) {
      LB_CUDA(cudaMemcpyAsync(probe, at<double2>(s, s->L.q0), bytes, cudaMemcpyDeviceToDevice, st), "probe states");
      LB_CUDA(cudaEventRecord(e0, st), "cudaEventRecord");
      r = propagate_impl(s, st, 0, 0, steps, probe, s->M);
      LB_CUDA(cudaEventRecord(e1, st), "cudaEventRecord");
    }
    if (r == LB_ECUDA) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return r;
    }
    if (r != LB_OK) continue;  // this candidate's inner solve does not converge here
    LB_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
    float ms = 0.0f;
    LB_CUDA(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    if (best < 0.0f || ms < best) {
      best = ms;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (win.sweep < 0) {
    s->rc = rc0;
    s->cluster = cl0;
    s->cc = cc0;
    s->method = s->hp.method = m0;
    s->hp.gM = gproj_used(s);
    s->hp.herm = use_symmetry(s) ? 1 : 0;
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
    return fail(LB_ENOTCONV, "no candidate's inner solve converged on the probe steps");
  }
  s->method = s->hp.method = win.method;
  s->cluster = win.sweep == LB_SWEEP_CLUSTER;
  s->cc = s->cluster ? cluster_cfg(s, win.E != 0) : cc0;
  s->hp.gM = gproj_used(s);
  s->hp.herm = use_symmetry(s) ? 1 : 0;
  if (win.sweep == LB_SWEEP_RESIDENT) {
    s->rc = lbk::resident_config(s->V, s->Q, n_coef(s), n_jcoef(s), s->N, s->jp.empty(), kry_elems(s));
    s->rc.E = win.E;
    s->rc.threads = ((s->V + win.E - 1) / win.E + 31) / 32 * 32;
    s->rc.QT = (win.E == 1 && s->Q <= 4 && s->jp.empty()) ? s->Q : 0;
  }
  LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
  LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (use_grid(s) && s->hp.pred_restart >= 0) {
    // the predictor's order: time the forward sweep over the first steps (at
    // least three rings' worth, so that the full order is reached) per order
    const int64_t pst = std::min<int64_t>(s->NT, std::max<int64_t>(probe_steps, 3 * lbk::kRingOrder));
    cudaEvent_t a = nullptr, b = nullptr;
    LB_CUDA(cudaEventCreate(&a), "cudaEventCreate");
    LB_CUDA(cudaEventCreate(&b), "cudaEventCreate");
    rc = ensure_ctab(s, st);
    if (rc) return rc;
    float tbest = -1.0f;
    int obest = s->pred_order;
    for (int o = 6; o <= lbk::kRingOrder; ++o) {
      s->hp.pred_order = o;
      LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
      LB_CUDA(cudaMemsetAsync(at<DevStatus>(s, s->L.status), 0, sizeof(DevStatus), st), "clear status");
      LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.gslots), 0, s->L.gslots.bytes, st), "clear grid slots");
      LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.bar), 0, s->L.bar.bytes, st), "clear grid barrier");
      LB_CUDA(cudaEventRecord(a, st), "cudaEventRecord");
      LB_CUDA(lbk::launch_sweep_grid(s->dp, 0, 1, 0, 0, pst, nullptr, s->M, s->gblocks, s->gsmem, s->hp.ff, st),
              "forward grid sweep");
      LB_CUDA(cudaEventRecord(b, st), "cudaEventRecord");
      DevStatus d{};
      LB_CUDA(cudaMemcpyAsync(&d, at<DevStatus>(s, s->L.status), sizeof(DevStatus), cudaMemcpyDeviceToHost, st),
              "read status");
      LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
      if (d.code) continue;
      float ms = 0.0f;
      LB_CUDA(cudaEventElapsedTime(&ms, a, b), "cudaEventElapsedTime");
      if (tbest < 0.0f || ms < tbest) {
        tbest = ms;
        obest = o;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    s->pred_order = obest;
    s->hp.pred_order = obest;
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
    LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  if (choice_out) {
    choice_out[0] = win.sweep;
    choice_out[1] = win.method;
    choice_out[2] = win.sweep == LB_SWEEP_RESIDENT ? s->rc.threads : (s->cluster ? s->cc.C : s->gblocks);
  }
  return LB_OK;
}

int lb_set_timing(lb_system* s, int32_t on) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (on && !s->ev[0])
    for (int i = 0; i < 4; ++i) LB_CUDA(cudaEventCreate(&s->ev[i]), "cudaEventCreate");
  s->timing = on != 0;
  return LB_OK;
}

int lb_controls_define(lb_system* s, int32_t n_splines, const int32_t* n_carriers, const double* carrier_ghz) {
  if (!s || !n_carriers || !carrier_ghz) return fail(LB_EINVAL, "null argument");
  if (s->ws) return fail(LB_EINVAL, "controls must be defined before binding a workspace");
  if (n_splines < 3) return fail(LB_EINVAL, "n_splines must be >= 3 (knot spacing T/(N_s-2))");
  int tot = 0;
  for (int q = 0; q < s->Q; ++q) {
    if (n_carriers[q] < 1 || n_carriers[q] > 64) return fail(LB_EINVAL, "n_carriers must be in 1..64");
    s->nf[q] = n_carriers[q];
    tot += n_carriers[q];
  }
  s->carriers.assign(tot, 0.0);
  for (int i = 0; i < tot; ++i) {
    if (!std::isfinite(carrier_ghz[i])) return fail(LB_EINVAL, "non-finite carrier frequency");
    s->carriers[i] = kTwoPi * carrier_ghz[i];
  }
  s->Ns = n_splines;
  s->n_params = 2 * n_splines * tot;
  s->alpha.assign(s->n_params, 0.0);
  s->ctrl_defined = true;
  s->ctab_dirty = true;
  return LB_OK;
}

int lb_controls_set_horizon(lb_system* s, double T_ns) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "set the control horizon before binding a workspace");
  if (!(T_ns >= 0.0) || !std::isfinite(T_ns)) return fail(LB_EINVAL, "the control horizon must be finite and >= 0");
  s->Tc = T_ns;
  s->ctab_dirty = true;
  return LB_OK;
}

int lb_controls_set(lb_system* s, const double* alpha, int64_t n) {
  if (!s || !alpha) return fail(LB_EINVAL, "null argument");
  if (!s->ctrl_defined) return fail(LB_EINVAL, "controls not defined");
  if (n != s->n_params) return fail(LB_EINVAL, "alpha length must be 2 * sum_q N_s N_f(q)");
  for (int64_t k = 0; k < n; ++k)
    if (!std::isfinite(alpha[k])) return fail(LB_EINVAL, "non-finite control coefficient");
  std::memcpy(s->alpha.data(), alpha, sizeof(double) * n);
  if (s->ws) return upload_controls(s, s->bind_stream);
  s->ctab_dirty = true;
  return LB_OK;
}

int lb_states_set(lb_system* s, int32_t M, const double* rho0, const double* weights) {
  if (!s || !rho0) return fail(LB_EINVAL, "null argument");
  if (M < 1) return fail(LB_EINVAL, "M must be >= 1");
  if (s->ws && M != s->Mu) return fail(LB_EINVAL, "M cannot change while a workspace is bound");
  std::vector<double> w(M, 1.0);
  if (weights)
    for (int i = 0; i < M; ++i) {
      if (!std::isfinite(weights[i])) return fail(LB_EINVAL, "non-finite weight");
      w[i] = weights[i];
    }
  for (int i = 0; i < M; ++i) w[i] /= (double)M;
  if (s->ws) {
    int rc = check_pairs(s, rho0, pairing_targets(s));
    if (rc) return rc;
  }
  if (s->Mu != M && s->target_mode == 1) s->target_mode = 0;  // explicit targets no longer match
  s->Mu = M;
  s->wgt_u = w;
  s->rho_herm = hermitian_matrices(rho0, M, s->N);
  s->rho_finite = true;
  for (size_t t = 0; t < (size_t)2 * M * s->N * s->N; ++t)
    if (!std::isfinite(rho0[t])) {
      s->rho_finite = false;
      break;
    }
  if (s->ws) {
    apply_pairs(s);
    int rc = upload_states(s, rho0, s->bind_stream);
    if (rc) return rc;
    if (s->target_mode == 2) {
      rc = upload_targets(s, s->bind_stream);
      if (rc) return rc;
    }
    return refresh_symmetry(s);
  }
  s->rho0.assign(rho0, rho0 + (size_t)2 * M * s->V);
  update_pairs(s);
  return LB_OK;
}

int lb_objective_set(lb_system* s, int32_t kind, const double* targets, double gamma2) {
  if (!s || !targets) return fail(LB_EINVAL, "null argument");
  if (kind != LB_J_FROB && kind != LB_J_TR) return fail(LB_EINVAL, "unknown merit functional");
  if (!(gamma2 >= 0.0) || !std::isfinite(gamma2)) return fail(LB_EINVAL, "gamma2 must be finite and >= 0");
  if (s->Mu < 1) return fail(LB_EINVAL, "call lb_states_set first");
  if (s->ws) {
    // the pairs are fixed while bound: these targets must not split them
    for (int u = 0; u < s->Mu; ++u) {
      const int e = s->pmap[u] >> 1, c = s->pmap[u] & 1;
      const size_t st = (size_t)2 * s->V;
      if (c && !is_conj_transpose(targets + s->evo[e] * st, targets + u * st, s->N))
        return fail(LB_EINVAL, "the targets split conjugate pairs of states the workspace was bound with (rebind)");
    }
  }
  s->kind = kind;
  s->gamma2 = gamma2;
  s->target_mode = 1;
  s->targets.assign(targets, targets + (size_t)2 * s->Mu * s->V);
  s->tar_herm = hermitian_matrices(targets, s->Mu, s->N);
  if (!s->ws) update_pairs(s);
  if (s->ws) {
    s->hp.kind = kind;
    s->hp.gamma2 = gamma2;
    s->hp.herm = use_symmetry(s) ? 1 : 0;
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, s->bind_stream), "upload problem");
    return upload_targets(s, s->bind_stream);
  }
  return LB_OK;
}

int lb_objective_set_measure(lb_system* s, int32_t m, double gamma2) {
  if (!s) return fail(LB_EINVAL, "null argument");
  if (m < 0 || m >= s->N) return fail(LB_EINVAL, "m must be in 0..N-1");
  if (!(gamma2 >= 0.0) || !std::isfinite(gamma2)) return fail(LB_EINVAL, "gamma2 must be finite and >= 0");
  if (s->Mu < 1) return fail(LB_EINVAL, "call lb_states_set first");
  if (s->ws && s->target_mode == 2) return fail(LB_EINVAL, "cannot leave a gate objective once a workspace is bound");
  // N_m as the (real, diagonal) target of every state
  std::vector<double> t((size_t)2 * s->Mu * s->V, 0.0);
  for (int i = 0; i < s->Mu; ++i)
    for (int l = 0; l < s->N; ++l) t[(size_t)2 * ((size_t)i * s->V + l + (size_t)s->N * l)] = std::abs(l - m);
  s->kind = LB_J_NM;
  s->gamma2 = gamma2;
  s->target_mode = 1;
  s->targets.swap(t);
  s->tar_herm = true;
  if (!s->ws) update_pairs(s);
  if (s->ws) {
    s->hp.kind = LB_J_NM;
    s->hp.gamma2 = gamma2;
    s->hp.herm = use_symmetry(s) ? 1 : 0;
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, s->bind_stream), "upload problem");
    return upload_targets(s, s->bind_stream);
  }
  return LB_OK;
}

int lb_objective_set_gate(lb_system* s, int32_t kind, const double* V, double gamma2) {
  if (!s || !V) return fail(LB_EINVAL, "null argument");
  if (kind != LB_J_FROB && kind != LB_J_TR) return fail(LB_EINVAL, "unknown merit functional");
  if (!(gamma2 >= 0.0) || !std::isfinite(gamma2)) return fail(LB_EINVAL, "gamma2 must be finite and >= 0");
  if (s->ws && s->target_mode != 2) return fail(LB_EINVAL, "switch to a gate objective before binding a workspace");
  s->kind = kind;
  s->gamma2 = gamma2;
  s->target_mode = 2;
  s->gateV.assign(V, V + (size_t)2 * s->Ne * s->Ne);
  s->targets.clear();
  s->tar_herm = true;
  if (!s->ws) update_pairs(s);
  if (s->ws) {
    s->hp.kind = kind;
    s->hp.gamma2 = gamma2;
    s->hp.herm = use_symmetry(s) ? 1 : 0;
    LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, s->bind_stream), "upload problem");
    return upload_targets(s, s->bind_stream);
  }
  return LB_OK;
}

int lb_solver_set(lb_system* s, int32_t method, double rtol, int32_t max_iter, int32_t ckpt_every) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "set the solver before binding a workspace");
  if (method == LB_SOLVER_AUTO) method = LB_SOLVER_JACOBI;
  if (method != LB_SOLVER_JACOBI && method != LB_SOLVER_NEUMANN && method != LB_SOLVER_GMRES)
    return fail(LB_EINVAL, "unknown solver");
  if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(LB_EINVAL, "rtol must be in (0, 1)");
  if (max_iter < 1 || max_iter > 100000) return fail(LB_EINVAL, "max_iter must be in 1..100000");
  if (ckpt_every < LB_CKPT_AUTO) return fail(LB_EINVAL, "ckpt_every must be >= 0 or LB_CKPT_AUTO");
  s->method = method;
  s->rtol = rtol;
  s->max_iter = max_iter;
  s->K = ckpt_every > s->NT ? (int)s->NT : ckpt_every;
  if (ckpt_every < 0) s->K = LB_CKPT_AUTO;
  return LB_OK;
}

int lb_system_set_coupling(lb_system* s, const double* jc_ghz, const double* rot_ghz) {
  if (!s || !jc_ghz) return fail(LB_EINVAL, "null argument");
  if (s->ws) return fail(LB_EINVAL, "set the coupling before binding a workspace");
  std::vector<int> jp, jq;
  std::vector<double> jg, je;
  for (int p = 0; p < s->Q; ++p)
    for (int q = p + 1; q < s->Q; ++q) {
      const double g = jc_ghz[p * s->Q + q];
      const double dr = rot_ghz ? rot_ghz[p] - rot_ghz[q] : 0.0;
      if (!std::isfinite(g) || !std::isfinite(dr)) return fail(LB_EINVAL, "non-finite coupling or frequency");
      if (g == 0.0) continue;
      jp.push_back(p);
      jq.push_back(q);
      jg.push_back(kTwoPi * g);
      je.push_back(kTwoPi * dr);
    }
  s->jp.swap(jp);
  s->jq.swap(jq);
  s->jg.swap(jg);
  s->je.swap(je);
  s->ctab_dirty = true;
  return LB_OK;
}

int lb_objective_set_penalty(lb_system* s, double gamma1, double a_ns) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "set the penalty before binding a workspace");
  if (!(gamma1 >= 0.0) || !std::isfinite(gamma1)) return fail(LB_EINVAL, "gamma1 must be finite and >= 0");
  if (!(a_ns > 0.0) || !std::isfinite(a_ns)) return fail(LB_EINVAL, "a must be finite and > 0");
  s->gamma1 = gamma1;
  s->pen_a = a_ns;
  return LB_OK;
}

int lb_set_symmetry(lb_system* s, int32_t symmetry) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (symmetry != LB_SYM_NONE && symmetry != LB_SYM_HERMITIAN && symmetry != LB_SYM_AUTO)
    return fail(LB_EINVAL, "unknown symmetry");
  s->symmetry = symmetry;
  return refresh_symmetry(s);
}

int lb_set_wait_limit(lb_system* s, int64_t polls) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (polls < 0) return fail(LB_EINVAL, "polls must be >= 0");
  s->spin_limit = polls;
  if (s->ws) {
    s->hp.spin_limit = polls;
    cudaStream_t st = s->bind_stream;
    LB_CUDA(cudaMemcpyAsync(&s->dp->spin_limit, &s->hp.spin_limit, sizeof(long long), cudaMemcpyHostToDevice, st),
            "upload wait limit");
    LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  return LB_OK;
}

int lb_set_difference_iterations(lb_system* s, int32_t on) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (on != 0 && on != 1) return fail(LB_EINVAL, "on must be 0 or 1");
  s->diffit = on;
  if (s->ws) {
    s->hp.diffit = on;
    cudaStream_t st = s->bind_stream;
    LB_CUDA(cudaMemcpyAsync(&s->dp->diffit, &s->hp.diffit, sizeof(int32_t), cudaMemcpyHostToDevice, st),
            "upload difference-iteration switch");
    LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  }
  return LB_OK;
}

int lb_set_precision(lb_system* s, int32_t precision) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "choose the precision before binding a workspace");
  if (precision != LB_PREC_F64 && precision != LB_PREC_F32X2) return fail(LB_EINVAL, "unknown precision");
  s->precision = precision;
  return LB_OK;
}

int lb_get_predictor(const lb_system* s, int32_t* restart, int32_t* order) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (restart) *restart = s->ws ? s->hp.pred_restart : effective_pred(s);
  if (order) *order = s->pred_order;
  return LB_OK;
}

int lb_set_pairing(lb_system* s, int32_t on) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "choose the pairing before binding a workspace");
  if (on != 0 && on != 1) return fail(LB_EINVAL, "pairing must be 0 or 1");
  s->pairing = on;
  update_pairs(s);
  return LB_OK;
}

int lb_set_predictor(lb_system* s, int32_t restart, int32_t order) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "set the predictor before binding a workspace");
  if (restart < LB_PRED_NONE) return fail(LB_EINVAL, "restart must be >= 0, LB_PRED_AUTO or LB_PRED_NONE");
  if (order < 0 || order > lbk::kRingOrder) return fail(LB_EINVAL, "order must be in 1..10 (0: the default, 8)");
  s->pred = restart;
  s->pred_order = order ? order : lbk::kDefaultRingOrder;
  return LB_OK;
}

int lb_set_sweep(lb_system* s, int32_t sweep) {
  if (!s) return fail(LB_EINVAL, "null system handle");
  if (s->ws) return fail(LB_EINVAL, "choose the sweep before binding a workspace");
  if (sweep != LB_SWEEP_AUTO && sweep != LB_SWEEP_RESIDENT && sweep != LB_SWEEP_GRID && sweep != LB_SWEEP_CLUSTER)
    return fail(LB_EINVAL, "unknown sweep kind");
  if (sweep == LB_SWEEP_CLUSTER && lbk::cluster_config(s->V, s->Q + (int)s->jp.size(), 1, 1, 1, false).C <= 0)
    return fail(LB_EINVAL, "cluster sweeps need Q + (Jaynes-Cummings pairs) <= 4 and N^2 * 2(Q + pairs) <= 1024");
  if (sweep == LB_SWEEP_RESIDENT && s->V > lbk::kMaxResidentV)
    return fail(LB_EINVAL, "one CTA per state needs N^2 <= 4096");
  s->sweep = sweep;
  return LB_OK;
}

int lb_workspace_bytes(const lb_system* s, size_t* bytes) {
  int rc = check_ready(s, false);
  if (rc) return rc;
  if (!bytes) return fail(LB_EINVAL, "null argument");
  *bytes = make_layout(s).total;
  return LB_OK;
}

int lb_bind_workspace(lb_system* s, void* ws, size_t bytes, void* stream) {
  int rc = check_ready(s, false);
  if (rc) return rc;
  if (!ws) return fail(LB_EINVAL, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(LB_EINVAL, "workspace must be 256-byte aligned");
  if (s->target_mode == 0) return fail(LB_EINVAL, "no objective (lb_objective_set or lb_objective_set_gate)");
  if (s->target_mode == 2) {
    for (int q = 0; q < s->Q; ++q)
      if (s->essential[q] < 1) return fail(LB_EINVAL, "bad essential levels");
  }
  rc = check_predictor(s);
  if (rc) return rc;
  s->L = make_layout(s);
  if (bytes < s->L.total) return fail(LB_ENOMEM, "workspace smaller than lb_workspace_bytes");
  s->tapes_packed = packed_tapes(s);
  if (s->rho0.empty()) return fail(LB_EINVAL, "initial states are required before binding");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = decide_krylov(s);
  if (rc) return rc;
  s->cluster = false;
  if (!use_grid(s) && s->sweep != LB_SWEEP_RESIDENT && s->method != LB_SOLVER_GMRES) {
    // 4Q lanes per element (shorter FP64 chain per iteration) when every
    // state's cluster still gets its own SMs, else 2Q lanes
    const lbk::ClusterConfig c1 = cluster_cfg(s, true), c0 = cluster_cfg(s, false);
    int dev = 0, nsm = 0;
    LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    LB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    const bool fit1 = c1.C > 0 && (long long)s->M * c1.C <= nsm, fit0 = c0.C > 0 && (long long)s->M * c0.C <= nsm;
    s->cc = fit1 ? c1 : c0;
    if (s->sweep == LB_SWEEP_CLUSTER) {
      if (s->cc.C <= 0) return fail(LB_EINVAL, "cluster sweeps need Q <= 4 and N^2 * 2Q <= 1024");
      s->cluster = true;
    } else {
      s->cluster = fit1 || fit0;
    }
  }
  if (use_grid(s)) {
    int dev = 0, coop = 0;
    LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    LB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "cudaDeviceGetAttribute");
    if (!coop) return fail(LB_ECUDA, "the device does not support cooperative launches (grid sweeps)");
    s->gsmem = lbk::grid_smem_bytes(n_coef(s), n_jcoef(s));
    const int ffk = s->precision == LB_PREC_F32X2 && s->jp.empty() ? 1 : 0;
    s->gblocks = lbk::grid_blocks(0, ffk, s->gsmem);
    s->gblocks_b = lbk::grid_blocks(1, ffk, s->gsmem);
    if (s->gblocks <= 0 || s->gblocks_b <= 0)
      return fail(LB_ECUDA, "cannot size the cooperative grid of the sweep kernels");
    if (s->gamma1 != 0.0 && !grid_chunks_cover_few_states(s))
      return fail(LB_EINVAL, "the running penalty on grid sweeps needs every block's elements to span at most "
                             "4 states (too many small states for the grid sweep)");
  }
  if (!s->upload_done) LB_CUDA(cudaEventCreateWithFlags(&s->upload_done, cudaEventDisableTiming), "cudaEventCreate");
  s->ws = static_cast<char*>(ws);
  s->ws_bytes = bytes;
  s->bind_stream = st;
  fill_prob(s);
  s->dp = at<ProbDev>(s, s->L.prob);
  s->d_items = at<WorkItem>(s, s->L.items);
  std::vector<WorkItem> items(s->M);
  for (int i = 0; i < s->M; ++i) items[i] = WorkItem{0, i};
  std::vector<double> sysp(4 * s->Q + s->Q * s->Q, 0.0);
  for (int q = 0; q < s->Q; ++q) {
    sysp[q] = s->det[q];
    sysp[s->Q + q] = s->kerr[q];
    sysp[2 * s->Q + s->Q * s->Q + q] = s->g1[q];
    sysp[3 * s->Q + s->Q * s->Q + q] = s->g2[q];
  }
  for (int i = 0; i < s->Q * s->Q; ++i) sysp[2 * s->Q + i] = s->xkerr[i];
  LB_CUDA(cudaMemsetAsync(s->ws, 0, s->L.total, st), "clear workspace");
  LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
  LB_CUDA(cudaMemcpyAsync(s->d_items, items.data(), sizeof(WorkItem) * s->M, cudaMemcpyHostToDevice, st),
          "upload work items");
  LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.sysp), sysp.data(), sizeof(double) * sysp.size(), cudaMemcpyHostToDevice,
                          st),
          "upload system");
  if (!s->carriers.empty())
    LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.carriers), s->carriers.data(), sizeof(double) * s->carriers.size(),
                            cudaMemcpyHostToDevice, st),
            "upload carriers");
  LB_CUDA(lbk::launch_tables(s->dp, s->hp, st), "tables kernel");
  rc = upload_symmetry_map(s, st);
  if (rc) return rc;
  rc = upload_states(s, s->rho0.data(), st);
  if (rc) return rc;
  rc = upload_targets(s, st);
  if (rc) return rc;
  rc = upload_controls(s, st);
  if (rc) return rc;
  LB_CUDA(cudaMemcpyAsync(at<int32_t>(s, s->L.pmap), s->pmap.data(), sizeof(int32_t) * s->Mu, cudaMemcpyHostToDevice,
                          st),
          "upload state pairs");
  s->rc = lbk::resident_config(s->V, s->Q, n_coef(s), n_jcoef(s), s->N, s->jp.empty(), kry_elems(s));
  // the workspace now owns the states; pageable copies above are staged
  s->rho0.clear();
  s->rho0.shrink_to_fit();
  return LB_OK;
}

static int run_forward(lb_system* s, cudaStream_t st, int tape) {
  NvtxRange nvtx("lb forward sweep");
  int rc = order_after_uploads(s, st);
  if (rc) return rc;
  s->launches = 0;
  rc = ensure_ctab(s, st);
  if (rc) return rc;
  LB_CUDA(cudaMemsetAsync(at<DevStatus>(s, s->L.status), 0, sizeof(DevStatus), st), "clear status");
  s->timed_fwd = s->timed_bwd = false;
  if (use_grid(s)) {
    LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.gslots), 0, s->L.gslots.bytes, st), "clear grid slots");
    LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.bar), 0, s->L.bar.bytes, st), "clear grid barrier");
    if (s->gamma1 != 0.0) LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.jpen), 0, s->L.jpen.bytes, st), "clear penalty");
    if (s->timing) LB_CUDA(cudaEventRecord(s->ev[0], st), "cudaEventRecord");
    LB_CUDA(lbk::launch_sweep_grid(s->dp, 0, 1, tape, 0, s->NT, nullptr, s->M, s->gblocks, s->gsmem, s->hp.ff, st),
            "forward grid sweep");
    if (s->timing) {
      LB_CUDA(cudaEventRecord(s->ev[1], st), "cudaEventRecord");
      s->timed_fwd = true;
    }
    LB_CUDA(lbk::launch_objective_states(s->dp, s->M, st), "objective kernel");
    s->launches += 2;
    return LB_OK;
  }
  if (s->timing) LB_CUDA(cudaEventRecord(s->ev[0], st), "cudaEventRecord");
  if (s->cluster)
    LB_CUDA(lbk::launch_forward_cluster(s->dp, s->M, tape, s->cc, st), "forward cluster kernel");
  else
    LB_CUDA(lbk::launch_forward_resident(s->dp, s->d_items, s->M, tape, s->rc, st), "forward kernel");
  if (s->timing) {
    LB_CUDA(cudaEventRecord(s->ev[1], st), "cudaEventRecord");
    s->timed_fwd = true;
  }
  s->launches += 1;
  return LB_OK;
}

static int finish(lb_system* s, cudaStream_t st, double* G_out, double* grad_out) {
  DevStatus d{};
  LB_CUDA(cudaMemcpyAsync(&d, at<DevStatus>(s, s->L.status), sizeof(DevStatus), cudaMemcpyDeviceToHost, st),
          "read status");
  double G = 0.0;
  if (G_out) LB_CUDA(cudaMemcpyAsync(&G, at<double>(s, s->L.G), sizeof(double), cudaMemcpyDeviceToHost, st), "read G");
  std::vector<double> g;
  if (grad_out) {
    g.resize(s->n_params);
    LB_CUDA(cudaMemcpyAsync(g.data(), at<double>(s, s->L.grad), sizeof(double) * s->n_params, cudaMemcpyDeviceToHost,
                            st),
            "read gradient");
  }
  LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  int rc = read_status(d, &s->last, s->launches);
  s->last.sweep = use_grid(s) ? LB_SWEEP_GRID : (s->cluster ? LB_SWEEP_CLUSTER : LB_SWEEP_RESIDENT);
  s->last.solver = s->method;
  s->last.ckpt_every = effective_K(s);
  s->last.symmetry = s->hp.herm ? LB_SYM_HERMITIAN : LB_SYM_NONE;
  s->last.states_integrated = s->M;
  if (s->timed_fwd) LB_CUDA(cudaEventElapsedTime(&s->last.ms_forward, s->ev[0], s->ev[1]), "cudaEventElapsedTime");
  if (s->timed_bwd) LB_CUDA(cudaEventElapsedTime(&s->last.ms_backward, s->ev[2], s->ev[3]), "cudaEventElapsedTime");
  if (rc) return rc;
  if (G_out) *G_out = G;
  if (grad_out) std::memcpy(grad_out, g.data(), sizeof(double) * s->n_params);
  return LB_OK;
}

int lb_forward(lb_system* s, void* stream, double* G_out, void* rhoT_dev_out) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = run_forward(s, st, 0);
  if (rc) return rc;
  LB_CUDA(lbk::launch_finalize(s->dp, 1, 0, 0, st), "objective kernel");
  s->launches += 1;
  if (rhoT_dev_out) {
    if (s->M == s->Mu) {
      LB_CUDA(cudaMemcpyAsync(rhoT_dev_out, at<double2>(s, s->L.qT), sizeof(double2) * (size_t)s->M * s->V,
                              cudaMemcpyDeviceToDevice, st),
              "copy final states");
    } else {
      // every given state: its integrated state or that state's conjugate transpose
      LB_CUDA(lbk::launch_expand_states(at<double2>(s, s->L.qT), at<int32_t>(s, s->L.pmap), s->Mu, s->N,
                                        static_cast<double2*>(rhoT_dev_out), st),
              "final states kernel");
      s->launches += 1;
    }
  }
  return finish(s, st, G_out, nullptr);
}

static int param_warps(const lb_system* s) {
  int nw = 0;
  for (int q = 0; q < s->Q; ++q) nw += s->nf[q] * s->Ns;
  return nw;
}

static int gradient_device(lb_system* s, cudaStream_t st) {
  int rc = run_forward(s, st, 1);
  if (rc) return rc;
  NvtxRange nvtx("lb recompute + adjoint sweep");
  if (use_grid(s)) {
    LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.gslots), 0, s->L.gslots.bytes, st), "clear grid slots");
    LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.bar), 0, s->L.bar.bytes, st), "clear grid barrier");
  }
  if (s->timing) LB_CUDA(cudaEventRecord(s->ev[2], st), "cudaEventRecord");
  if (use_grid(s))
    LB_CUDA(lbk::launch_backward_grid(s->dp, s->gblocks_b, s->gsmem, s->hp.ff, st), "backward grid sweep");
  else if (s->cluster)
    LB_CUDA(lbk::launch_backward_cluster(s->dp, s->M, s->cc, st), "backward cluster kernel");
  else
    LB_CUDA(lbk::launch_backward_resident(s->dp, s->d_items, s->M, s->rc, st), "backward kernel");
  if (s->timing) {
    LB_CUDA(cudaEventRecord(s->ev[3], st), "cudaEventRecord");
    s->timed_bwd = true;
  }
  LB_CUDA(lbk::launch_finalize(s->dp, 1, param_warps(s), 1, st), "finalize kernels");
  s->launches += 4;  // backward sweep, objective, slot sum, projection
  return LB_OK;
}

int lb_gradient(lb_system* s, void* stream, double* G_out, double* grad_out) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = gradient_device(s, st);
  if (rc) return rc;
  return finish(s, st, G_out, grad_out);
}

namespace {

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double t = 0.0;
  for (size_t i = 0; i < a.size(); ++i) t += a[i] * b[i];
  return t;
}
double max_abs(const std::vector<double>& a) {
  double t = 0.0;
  for (double v : a) t = std::max(t, std::fabs(v));
  return t;
}

// d = -H g by the two-loop recursion over the pairs (S[k], Y[k]), oldest
// first; with no pair, -g scaled to max-norm step0.
void lbfgs_direction(const std::vector<double>& g, const std::vector<std::vector<double>>& S,
                     const std::vector<std::vector<double>>& Y, double step0, std::vector<double>& d) {
  const size_t n = g.size(), m = S.size();
  d.assign(n, 0.0);
  if (m == 0) {
    const double sc = step0 / max_abs(g);
    for (size_t i = 0; i < n; ++i) d[i] = -g[i] * sc;
    return;
  }
  std::vector<double> q = g, rho(m), a(m);
  for (size_t k = m; k-- > 0;) {
    rho[k] = 1.0 / dot(Y[k], S[k]);
    a[k] = rho[k] * dot(S[k], q);
    for (size_t i = 0; i < n; ++i) q[i] -= a[k] * Y[k][i];
  }
  const double gamma = dot(S[m - 1], Y[m - 1]) / dot(Y[m - 1], Y[m - 1]);
  for (size_t i = 0; i < n; ++i) q[i] *= gamma;
  for (size_t k = 0; k < m; ++k) {
    const double b = rho[k] * dot(Y[k], q);
    for (size_t i = 0; i < n; ++i) q[i] += (a[k] - b) * S[k][i];
  }
  for (size_t i = 0; i < n; ++i) d[i] = -q[i];
}

}  // namespace

int lb_optimize(lb_system* s, void* stream, int32_t max_iter, int32_t memory, double gtol, double step0,
                double* G_out, double* alpha_out, int32_t* iters_out, int32_t* evals_out, double* history) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  if (memory < 1 || max_iter < 0 || !(gtol >= 0.0) || !(step0 > 0.0) || !std::isfinite(step0))
    return fail(LB_EINVAL, "need memory >= 1, max_iter >= 0, gtol >= 0 and step0 > 0");
  NvtxRange nvtx("lb_optimize");
  const size_t n = (size_t)s->n_params;
  constexpr double kC1 = 1e-4, kCurv = 1e-10;
  constexpr int kMaxTrials = 30;
  std::vector<double> x = s->alpha, g(n), xn(n), gn(n), d;
  std::vector<std::vector<double>> S, Y;
  double f = 0.0;
  rc = lb_gradient(s, stream, &f, g.data());
  if (rc) return rc;
  int evals = 1, iters = 0;
  if (history) {
    history[0] = f;
    history[1] = max_abs(g);
  }
  for (; iters < max_iter; ++iters) {
    if (max_abs(g) <= gtol) break;
    lbfgs_direction(g, S, Y, step0, d);
    double gd = dot(g, d);
    if (!(gd < 0.0)) {
      S.clear();
      Y.clear();
      lbfgs_direction(g, S, Y, step0, d);
      gd = dot(g, d);
    }
    double t = 1.0, fn = 0.0;
    bool accepted = false;
    for (int trial = 0; trial < kMaxTrials; ++trial) {
      for (size_t i = 0; i < n; ++i) xn[i] = x[i] + t * d[i];
      rc = lb_controls_set(s, xn.data(), (int64_t)n);
      if (rc) return rc;
      rc = lb_gradient(s, stream, &fn, gn.data());
      ++evals;
      if (rc) return rc;
      if (fn <= f + kC1 * t * gd) {
        accepted = true;
        break;
      }
      t *= 0.5;
    }
    if (!accepted) {
      // no sufficient decrease along d: stop at the current iterate
      rc = lb_controls_set(s, x.data(), (int64_t)n);
      if (rc) return rc;
      break;
    }
    std::vector<double> sv(n), yv(n);
    for (size_t i = 0; i < n; ++i) {
      sv[i] = xn[i] - x[i];
      yv[i] = gn[i] - g[i];
    }
    if (dot(sv, yv) > kCurv * std::sqrt(dot(sv, sv)) * std::sqrt(dot(yv, yv))) {
      S.push_back(std::move(sv));
      Y.push_back(std::move(yv));
      if ((int)S.size() > memory) {
        S.erase(S.begin());
        Y.erase(Y.begin());
      }
    }
    x = xn;
    g = gn;
    f = fn;
    if (history) {
      history[2 * (iters + 1)] = f;
      history[2 * (iters + 1) + 1] = max_abs(g);
    }
  }
  if (G_out) *G_out = f;
  if (alpha_out) std::memcpy(alpha_out, x.data(), sizeof(double) * n);
  if (iters_out) *iters_out = iters;
  if (evals_out) *evals_out = evals;
  return LB_OK;
}

int lb_gradient_async(lb_system* s, void* stream, void* G_dev, void* grad_dev) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = gradient_device(s, st);
  if (rc) return rc;
  if (G_dev)
    LB_CUDA(cudaMemcpyAsync(G_dev, at<double>(s, s->L.G), sizeof(double), cudaMemcpyDeviceToDevice, st), "copy G");
  if (grad_dev)
    LB_CUDA(cudaMemcpyAsync(grad_dev, at<double>(s, s->L.grad), sizeof(double) * s->n_params, cudaMemcpyDeviceToDevice,
                            st),
            "copy gradient");
  return LB_OK;
}

static int propagate_impl(lb_system* s, cudaStream_t st, int adjoint, int64_t j0, int64_t j1, double2* x, int n_vec) {
  int rc = order_after_uploads(s, st);
  if (rc) return rc;
  s->launches = 0;
  rc = ensure_ctab(s, st);
  if (rc) return rc;
  LB_CUDA(cudaMemsetAsync(at<DevStatus>(s, s->L.status), 0, sizeof(DevStatus), st), "clear status");
  s->timed_fwd = s->timed_bwd = false;
  if (j1 > j0) {
    if (use_grid(s)) {
      if (n_vec > s->M) return fail(LB_EINVAL, "grid sweeps propagate at most M vectors at a time");
      LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.gslots), 0, s->L.gslots.bytes, st), "clear grid slots");
      LB_CUDA(cudaMemsetAsync(at<char>(s, s->L.bar), 0, s->L.bar.bytes, st), "clear grid barrier");
      LB_CUDA(lbk::launch_sweep_grid(s->dp, adjoint ? 2 : 1, 0, 0, j0, j1, x, n_vec, s->gblocks, s->gsmem, s->hp.ff, st),
              "propagate grid sweep");
    } else if (s->cluster) {
      LB_CUDA(lbk::launch_propagate_cluster(s->dp, adjoint, j0, j1, x, n_vec, s->cc, st), "propagate cluster kernel");
    } else {
      LB_CUDA(lbk::launch_propagate_resident(s->dp, adjoint, j0, j1, x, n_vec, s->rc, st), "propagate kernel");
    }
    s->launches += 1;
  }
  return finish(s, st, nullptr, nullptr);
}

int lb_propagate(lb_system* s, void* stream, int32_t adjoint, int64_t j0, int64_t j1, void* x_dev, int32_t n_vec) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  if (!x_dev || n_vec < 1) return fail(LB_EINVAL, "bad vectors");
  if (j0 < 0 || j1 < j0 || j1 > s->NT) return fail(LB_EINVAL, "need 0 <= j0 <= j1 <= n_steps");
  return propagate_impl(s, static_cast<cudaStream_t>(stream), adjoint, j0, j1, static_cast<double2*>(x_dev), n_vec);
}

int lb_apply(lb_system* s, void* stream, int32_t adjoint, int64_t step, const void* x_dev, void* y_dev,
             int32_t n_vec) {
  int rc = check_ready(s, true);
  if (rc) return rc;
  if (!x_dev || !y_dev || n_vec < 1) return fail(LB_EINVAL, "bad vectors");
  if (step < 0 || step >= s->NT) return fail(LB_EINVAL, "step out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = order_after_uploads(s, st);
  if (rc) return rc;
  rc = ensure_ctab(s, st);
  if (rc) return rc;
  LB_CUDA(lbk::launch_apply(s->dp, s->hp, adjoint, step, static_cast<const double2*>(x_dev), static_cast<double2*>(y_dev),
                            n_vec, st),
          "apply kernel");
  return LB_OK;
}

int lb_get_stats(lb_system* s, lb_stats* out) {
  if (!s || !out) return fail(LB_EINVAL, "null argument");
  *out = s->last;
  return LB_OK;
}

// ---------------------------------------------------------------------------
// batches

int lb_batch_create(lb_system* const* systems, int32_t n, lb_batch** out) {
  if (!systems || n < 1 || !out) return fail(LB_EINVAL, "bad batch arguments");
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return fail(LB_ENOMEM, "host allocation failed");
  int maxV = 0, maxQ = 0, maxc = 0, maxj = 0, maxN = 0, minQ = LB_MAXQ + 1;
  size_t maxkry = 0;
  bool pairs = false;
  for (int i = 0; i < n; ++i) {
    lb_system* s = systems[i];
    if (!s || !s->ws) {
      delete b;
      return fail(LB_EINVAL, "every system of a batch must have a bound workspace");
    }
    if (use_grid(s)) {
      delete b;
      return fail(LB_EINVAL, "batched systems must use one CTA per state (N^2 <= 4096, LB_SWEEP_RESIDENT)");
    }
    b->sys.push_back(s);
    b->grad_off.push_back(b->n_grad);
    b->n_grad += s->n_params;
    b->n_items += s->M;
    maxV = std::max(maxV, s->V);
    maxQ = std::max(maxQ, s->Q);
    minQ = std::min(minQ, s->Q);
    maxc = std::max(maxc, n_coef(s));
    maxj = std::max(maxj, n_jcoef(s));
    maxN = std::max(maxN, s->N);
    maxkry = std::max(maxkry, kry_elems(s));
    pairs = pairs || !s->jp.empty();
    b->max_param_warps = std::max(b->max_param_warps, param_warps(s));
  }
  b->rc = lbk::resident_config(maxV, maxQ, maxc, maxj, maxN, minQ == maxQ && !pairs, maxkry);
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    delete b;
    return fail(LB_ECUDA, "cannot read the device's shared memory limit");
  }
  if (b->rc.smem > (size_t)optin) {
    delete b;
    return fail(LB_EINVAL, "the batch's largest state and GMRES basis do not fit one CTA's shared memory together");
  }
  *out = b;
  return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  for (int m = 0; m < 2; ++m) {
    if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
    if (b->graph[m]) cudaGraphDestroy(b->graph[m]);
  }
  delete b;
}

static size_t batch_layout(const lb_batch* b, size_t* o_probs, size_t* o_items, size_t* o_goff, size_t* o_G,
                           size_t* o_grad, size_t* o_st) {
  const size_t n = b->sys.size();
  size_t off = 0;
  *o_probs = off;
  off += align_up(sizeof(ProbDev) * n);
  *o_items = off;
  off += align_up(sizeof(WorkItem) * b->n_items);
  *o_goff = off;
  off += align_up(sizeof(int64_t) * n);
  *o_G = off;
  off += align_up(sizeof(double) * n);
  *o_grad = off;
  off += align_up(sizeof(double) * (b->n_grad ? b->n_grad : 1));
  *o_st = off;
  off += align_up(sizeof(DevStatus) * n);
  return off;
}

int lb_batch_workspace_bytes(const lb_batch* b, size_t* bytes) {
  if (!b || !bytes) return fail(LB_EINVAL, "null argument");
  size_t a, c, d, e, f, g;
  *bytes = batch_layout(b, &a, &c, &d, &e, &f, &g);
  return LB_OK;
}

int lb_batch_bind_workspace(lb_batch* b, void* ws, size_t bytes, void* stream) {
  if (!b || !ws) return fail(LB_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(LB_EINVAL, "workspace must be 256-byte aligned");
  size_t o_probs, o_items, o_goff, o_G, o_grad, o_st;
  const size_t need = batch_layout(b, &o_probs, &o_items, &o_goff, &o_G, &o_grad, &o_st);
  if (bytes < need) return fail(LB_ENOMEM, "batch workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  b->ws = base;
  b->ws_bytes = bytes;
  b->d_probs = reinterpret_cast<ProbDev*>(base + o_probs);
  b->d_items = reinterpret_cast<WorkItem*>(base + o_items);
  b->d_grad_off = reinterpret_cast<int64_t*>(base + o_goff);
  b->d_G = reinterpret_cast<double*>(base + o_G);
  b->d_grad = reinterpret_cast<double*>(base + o_grad);
  b->d_st = reinterpret_cast<DevStatus*>(base + o_st);
  std::vector<ProbDev> probs;
  // work items, most expensive first (cost ~ V * Q per state-step)
  std::vector<std::pair<double, WorkItem>> order;
  for (size_t p = 0; p < b->sys.size(); ++p) {
    lb_system* s = b->sys[p];
    probs.push_back(s->hp);
    for (int i = 0; i < s->M; ++i)
      order.push_back({-(double)s->V * (s->Q + 1) * (double)s->NT, WorkItem{(int32_t)p, i}});
    // the systems' own uploads must precede the batch's work
    int rc = order_after_uploads(s, st);
    if (rc) return rc;
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<double, WorkItem>& x, const std::pair<double, WorkItem>& y) {
                     return x.first < y.first;
                   });
  std::vector<WorkItem> items;
  for (auto& o : order) items.push_back(o.second);
  LB_CUDA(cudaMemcpyAsync(b->d_probs, probs.data(), sizeof(ProbDev) * probs.size(), cudaMemcpyHostToDevice, st),
          "upload batch problems");
  LB_CUDA(cudaMemcpyAsync(b->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice, st),
          "upload batch items");
  LB_CUDA(cudaMemcpyAsync(b->d_grad_off, b->grad_off.data(), sizeof(int64_t) * b->grad_off.size(),
                          cudaMemcpyHostToDevice, st),
          "upload gradient offsets");
  LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  return LB_OK;
}

// device work of one batch call (graph-capturable: no host synchronisation)
static int batch_enqueue(lb_batch* b, cudaStream_t st, int with_grad) {
  NvtxRange nvtx(with_grad ? "lb batch gradient" : "lb batch forward");
  for (lb_system* s : b->sys) {
    LB_CUDA(lbk::launch_control_table(s->dp, s->hp, st), "control table kernel");
    s->ctab_dirty = false;
    LB_CUDA(cudaMemsetAsync(s->hp.status, 0, sizeof(DevStatus), st), "clear status");
  }
  LB_CUDA(lbk::launch_forward_resident(b->d_probs, b->d_items, b->n_items, with_grad, b->rc, st), "forward kernel");
  if (with_grad)
    LB_CUDA(lbk::launch_backward_resident(b->d_probs, b->d_items, b->n_items, b->rc, st), "backward kernel");
  LB_CUDA(lbk::launch_finalize(b->d_probs, (int)b->sys.size(), b->max_param_warps, with_grad, st), "finalize kernels");
  LB_CUDA(lbk::launch_gather(b->d_probs, (int)b->sys.size(), b->d_grad_off, b->d_G, with_grad ? b->d_grad : nullptr,
                             b->d_st, st),
          "gather kernel");
  return LB_OK;
}

static int batch_call(lb_batch* b, cudaStream_t st, int with_grad, double* G_out, double* grad_out) {
  if (!b->ws) return fail(LB_EINVAL, "no batch workspace bound");
  const int mode = with_grad ? 1 : 0;
  for (lb_system* s : b->sys) {
    int rc = order_after_uploads(s, st);
    if (rc) return rc;
  }
  int launches = 0;
  if (b->exec[mode]) {
    LB_CUDA(cudaGraphLaunch(b->exec[mode], st), "cudaGraphLaunch");
    launches = 2 * (int)b->sys.size() + 3 + 3 * with_grad;
  } else {
    int rc = batch_enqueue(b, st, with_grad);
    if (rc) return rc;
    launches = 2 * (int)b->sys.size() + 3 + 3 * with_grad;
  }
  const size_t n = b->sys.size();
  std::vector<DevStatus> stv(n);
  LB_CUDA(cudaMemcpyAsync(stv.data(), b->d_st, sizeof(DevStatus) * n, cudaMemcpyDeviceToHost, st), "read status");
  std::vector<double> G(n), g;
  if (G_out) LB_CUDA(cudaMemcpyAsync(G.data(), b->d_G, sizeof(double) * n, cudaMemcpyDeviceToHost, st), "read G");
  if (grad_out && with_grad) {
    g.resize(b->n_grad);
    LB_CUDA(cudaMemcpyAsync(g.data(), b->d_grad, sizeof(double) * b->n_grad, cudaMemcpyDeviceToHost, st),
            "read gradients");
  }
  LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  lb_stats tot{};
  for (size_t p = 0; p < n; ++p) {
    lb_stats one{};
    int rc = read_status(stv[p], &one, 0);
    if (rc) {
      g_err = "system " + std::to_string(p) + ": " + g_err;
      return rc;
    }
    tot.state_steps += one.state_steps;
    tot.inner_iterations += one.inner_iterations;
    for (int ph = 0; ph < 3; ++ph) {
      tot.phase_steps[ph] += one.phase_steps[ph];
      tot.phase_iterations[ph] += one.phase_iterations[ph];
      tot.phase_diff_iterations[ph] += one.phase_diff_iterations[ph];
    }
    tot.max_iterations = std::max(tot.max_iterations, one.max_iterations);
  }
  tot.kernel_launches = launches;
  b->last = tot;
  if (G_out) std::memcpy(G_out, G.data(), sizeof(double) * n);
  if (grad_out && with_grad) std::memcpy(grad_out, g.data(), sizeof(double) * b->n_grad);
  return LB_OK;
}

int lb_batch_forward(lb_batch* b, void* stream, double* G_out) {
  if (!b) return fail(LB_EINVAL, "null batch");
  return batch_call(b, static_cast<cudaStream_t>(stream), 0, G_out, nullptr);
}

int lb_batch_gradient(lb_batch* b, void* stream, double* G_out, double* grad_out) {
  if (!b) return fail(LB_EINVAL, "null batch");
  return batch_call(b, static_cast<cudaStream_t>(stream), 1, G_out, grad_out);
}

int lb_batch_capture_graph(lb_batch* b, void* stream, int32_t mode) {
  if (!b) return fail(LB_EINVAL, "null batch");
  if (mode == -1) {
    for (int m = 0; m < 2; ++m) {
      if (b->exec[m]) cudaGraphExecDestroy(b->exec[m]);
      if (b->graph[m]) cudaGraphDestroy(b->graph[m]);
      b->exec[m] = nullptr;
      b->graph[m] = nullptr;
    }
    return LB_OK;
  }
  if (mode != 0 && mode != 1) return fail(LB_EINVAL, "mode must be 0, 1 or -1");
  if (!b->ws) return fail(LB_EINVAL, "no batch workspace bound");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return fail(LB_EINVAL, "graph capture needs a non-default stream");
  for (lb_system* s : b->sys) {
    int rc = order_after_uploads(s, st);
    if (rc) return rc;
  }
  LB_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  if (b->exec[mode]) cudaGraphExecDestroy(b->exec[mode]);
  if (b->graph[mode]) cudaGraphDestroy(b->graph[mode]);
  b->exec[mode] = nullptr;
  b->graph[mode] = nullptr;
  LB_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  int rc = batch_enqueue(b, st, mode);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  b->graph[mode] = g;
  LB_CUDA(cudaGraphInstantiate(&b->exec[mode], g, 0), "cudaGraphInstantiate");
  return LB_OK;
}

int lb_batch_get_stats(lb_batch* b, lb_stats* out) {
  if (!b || !out) return fail(LB_EINVAL, "null argument");
  *out = b->last;
  return LB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Gradient with the device scratch in a static array (no device allocation)
//
// For callers that cannot allocate device memory at all: code that runs where
// cudaMalloc is not allowed or not wanted (inside a host callback, inside a
// framework that owns every byte of device memory, or in a control loop that
// must not touch the allocator).  Everything the call needs on the device
// lives in g_lb_static_scratch, a file-scope array that every GPU loading this
// library holds until the process exits.

static __device__ __align__(256) unsigned char g_lb_static_scratch[LB_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices] = {};  // device address of the array, per device

// Device address of g_lb_static_scratch on the current device.  In host code
// the array's name only denotes a host-side stand-in, so the address is looked
// up with that device current.  Outside a stream capture it is looked up on
// every call (cheap once the module is loaded, and right again after a
// cudaDeviceReset has reloaded the module); during a capture the address the
// last call outside one found is used.
int static_scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  LB_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxStaticDevices) return fail(LB_EINVAL, "device ordinal too large for the static scratch");
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  LB_CUDA(cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_static_ptr[dev]) {
    void* p = nullptr;
    LB_CUDA(cudaGetSymbolAddress(&p, g_lb_static_scratch), "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return LB_OK;
}

// Upload the handle's host-side inputs into the static scratch, like
// lb_bind_workspace, but keep the host copies: the array is shared by every
// call, so each call uploads everything again.
int static_bind(lb_system* s, void* ws, cudaStream_t st) {
  int rc0 = decide_krylov(s);
  if (rc0) return rc0;
  s->cluster = false;  // this entry point always runs one CTA per state
  s->L = make_layout(s);
  s->tapes_packed = packed_tapes(s);
  s->ws = static_cast<char*>(ws);
  s->ws_bytes = LB_STATIC_SCRATCH_BYTES;
  s->bind_stream = st;
  fill_prob(s);
  s->dp = at<ProbDev>(s, s->L.prob);
  s->d_items = at<WorkItem>(s, s->L.items);
  std::vector<WorkItem> items(s->M);
  for (int i = 0; i < s->M; ++i) items[i] = WorkItem{0, i};
  std::vector<double> sysp(4 * s->Q + s->Q * s->Q, 0.0);
  for (int q = 0; q < s->Q; ++q) {
    sysp[q] = s->det[q];
    sysp[s->Q + q] = s->kerr[q];
    sysp[2 * s->Q + s->Q * s->Q + q] = s->g1[q];
    sysp[3 * s->Q + s->Q * s->Q + q] = s->g2[q];
  }
  for (int i = 0; i < s->Q * s->Q; ++i) sysp[2 * s->Q + i] = s->xkerr[i];
  // the array keeps the previous call's contents: clear all of it
  LB_CUDA(cudaMemsetAsync(s->ws, 0, s->L.total, st), "clear static scratch");
  LB_CUDA(cudaMemcpyAsync(s->dp, &s->hp, sizeof(ProbDev), cudaMemcpyHostToDevice, st), "upload problem");
  LB_CUDA(cudaMemcpyAsync(s->d_items, items.data(), sizeof(WorkItem) * s->M, cudaMemcpyHostToDevice, st),
          "upload work items");
  LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.sysp), sysp.data(), sizeof(double) * sysp.size(), cudaMemcpyHostToDevice,
                          st),
          "upload system");
  if (!s->carriers.empty())
    LB_CUDA(cudaMemcpyAsync(at<double>(s, s->L.carriers), s->carriers.data(), sizeof(double) * s->carriers.size(),
                            cudaMemcpyHostToDevice, st),
            "upload carriers");
  LB_CUDA(lbk::launch_tables(s->dp, s->hp, st), "tables kernel");
  int rc = upload_symmetry_map(s, st);
  if (rc) return rc;
  rc = upload_states(s, s->rho0.data(), st);
  if (rc) return rc;
  rc = upload_targets(s, st);
  if (rc) return rc;
  rc = upload_controls(s, st);
  if (rc) return rc;
  LB_CUDA(cudaMemcpyAsync(at<int32_t>(s, s->L.pmap), s->pmap.data(), sizeof(int32_t) * s->Mu, cudaMemcpyHostToDevice,
                          st),
          "upload state pairs");
  s->rc = lbk::resident_config(s->V, s->Q, n_coef(s), n_jcoef(s), s->N, s->jp.empty(), kry_elems(s));
  return LB_OK;
}

// Leave the handle unbound again, whatever happened; once device work has
// been queued, wait for it on every exit path (an early error return
// included), so that nothing of this call still writes the shared array when
// the caller gets control back.
struct StaticUnbind {
  lb_system* s;
  cudaStream_t st;
  bool queued = false;
  ~StaticUnbind() {
    if (queued) (void)cudaStreamSynchronize(st);
    s->ws = nullptr;
    s->ws_bytes = 0;
    s->dp = nullptr;
    s->d_items = nullptr;
    s->bind_stream = nullptr;
    s->ctab_dirty = true;
  }
};

}  // namespace

extern "C" int lb_gradient_static(lb_system* s, void* stream, double* G_out, double* grad_out) {
  int rc = check_ready(s, false);
  if (rc) return rc;
  if (s->ws) return fail(LB_EINVAL, "lb_gradient_static needs a handle without a bound workspace");
  if (use_grid(s)) return fail(LB_EINVAL, "lb_gradient_static supports one CTA per state only (N^2 <= 4096)");
  if (s->sweep == LB_SWEEP_CLUSTER)
    return fail(LB_EINVAL, "lb_gradient_static runs one CTA per state; LB_SWEEP_CLUSTER is not available there");
  rc = check_predictor(s);
  if (rc) return rc;
  if (s->target_mode == 0) return fail(LB_EINVAL, "no objective (lb_objective_set or lb_objective_set_gate)");
  if (s->rho0.empty()) return fail(LB_EINVAL, "no initial states");
  const size_t need = make_layout(s).total;
  if (need > (size_t)LB_STATIC_SCRATCH_BYTES) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "problem needs %zu bytes of device scratch; the static scratch holds %zu",
                  need, (size_t)LB_STATIC_SCRATCH_BYTES);
    return fail(LB_ENOMEM, buf);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* ws = nullptr;
  rc = static_scratch_address(st, &ws);
  if (rc) return rc;
  StaticUnbind guard{s, st};
  guard.queued = true;
  rc = static_bind(s, ws, st);
  if (rc) return rc;
  rc = gradient_device(s, st);
  if (rc) return rc;
  return finish(s, st, G_out, grad_out);
}
