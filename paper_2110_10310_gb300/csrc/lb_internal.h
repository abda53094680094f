// Internal declarations shared by the host library and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "lindblad_gb300.h"

#define LB_MAXQ LB_MAX_SUBSYSTEMS
#define LB_MAXN LB_MAX_LEVELS

// Status block written by the kernels and read by the host after a sync.
struct DevStatus {
  int32_t code;                 // 0 or LB_ENOTCONV / LB_ENAN (first error wins)
  int32_t step;                 // time step of the first error
  int32_t max_iter_seen;        // largest iteration count of one step
  int32_t pad;
  unsigned long long iters[3];  // iterations per phase: forward, recompute, adjoint
  unsigned long long steps[3];  // state-steps per phase
  unsigned long long diters[3]; // of iters: difference iterations in single precision (grid sweeps)
};

// Grid-wide barrier state of a cooperative launch (zeroed before each launch).
struct GridBar {
  unsigned int count;  // blocks arrived in the current generation
  unsigned int gen;    // generation counter
  int err;             // set when a wait gave up
  int pad;
};

// Everything a kernel needs to know about one system, in device memory.
// Arrays are device pointers into the system's workspace.
struct ProbDev {
  int32_t Q, N, M, NT;
  int32_t V;  // N*N (N <= 2^15 keeps V and all element offsets in 32 bits per state)
  int32_t K;  // checkpoint interval; 0 = keep every stage vector z^j
  int32_t n_ckpt, max_iter, method, kind;
  int32_t Ns, n_params;
  int32_t krylov;            // GMRES cycle length m (Krylov basis of m + 1 vectors in shared memory)
  int32_t dbits;             // bits per packed digit: ceil(log2 max n_q), at least 4
  int32_t npair;             // Jaynes-Cummings pairs p < q with g_pq != 0
  int32_t cq;                // entries per step of ctab: Q control factors, then npair coupling factors
  int32_t jp[LB_MAXQ * (LB_MAXQ - 1) / 2], jq[LB_MAXQ * (LB_MAXQ - 1) / 2];
  double jg[LB_MAXQ * (LB_MAXQ - 1) / 2];  // g_pq (rad/ns)
  double je[LB_MAXQ * (LB_MAXQ - 1) / 2];  // eta_pq = omega_p^rot - omega_q^rot (rad/ns)
  double h, rtol, T, gamma2;
  double Tc;                 // horizon the B-splines span (knot spacing Tc / (Ns - 2))
  int32_t levels[LB_MAXQ];
  int32_t stride[LB_MAXQ];   // s_q = prod_{p>q} n_p
  int32_t coff[LB_MAXQ];     // offset of subsystem q in cu/cd
  int32_t joff[LB_MAXQ];     // offset of subsystem q in jf/ja
  int32_t nf[LB_MAXQ];       // carriers per subsystem
  int32_t foff[LB_MAXQ];     // offset of subsystem q in carriers
  int32_t aoff[LB_MAXQ];     // offset of subsystem q in alpha
  double jump[LB_MAXQ];      // (dt/2)/T1_q, 0 = no decay
  int32_t ncoef, njcoef;     // sizes of cu/cd and jf/ja
  // system parameters: det[Q], kerr[Q] (rad/ns), xkerr[Q*Q] (rad/ns, p<q used),
  // g1[Q] = 1/T1, g2[Q] = 1/T2 (1/ns, 0 = off)
  double* sysp;
  // time-independent tables
  double* cu;                // [ncoef]  sqrt(n+1) if n+1 < n_q else 0
  double* cd;                // [ncoef]  sqrt(n)
  double* jf;                // [njcoef] jump_q sqrt((nk+1)(nl+1)), 0 if a digit would leave the range
  double* ja;                // [njcoef] jump_q sqrt(nk nl)
  uint32_t* digits;          // [N] digits of a basis index, subsystem q at bits dbits q .. dbits (q + 1) - 1
  double2* D;                // [V] diagonal of M
  double2* Dinv;             // [V] 1/(1 - dt/2 D)
  // controls
  double* alpha;             // [n_params]
  double* carriers;          // [sum nf] Omega (rad/ns)
  double2* ctab;             // [NT][cq] (dt/2) d_q(t_j + dt/2), then (dt/2) g_pq e^{i eta_pq (t_j + dt/2)}
  double* sfac;              // [NT] factor of the inner stopping test per step (k_stop_factors)
  double* pen;               // [NT] running-penalty weights dt beta(t_j) (gamma1 != 0)
  double2* qb;               // [M*V] q^j rebuilt backwards in the adjoint sweep (gamma1 != 0)
  double* jpen;              // [M] grid sweeps: sum_j dt beta(t_j) J(q^j) per state (gamma1 != 0)
  double* mpart;             // [grid_blocks][4] grid sweeps: per-block merit sums of one step (gamma1 != 0)
  double gamma1, pen_a;      // running-penalty weight and width a (ns)
  // states and objective
  double2* q0;               // [M*V]
  double2* tar;              // [M*V]
  double* wgt;               // [M] beta_i / M
  double2* qT;               // [M*V]
  double2* ckpt;             // [M*n_ckpt*V], or [M*NT*V] of z^j when K == 0
  double2* seg;              // [M*K*V] stage vectors of one segment (K > 0)
  double2* gproj;            // [gM][NT][Q][2] per slot/step: g_a, g_ad (eq. reducedgradient pieces)
  double2* gsum;             // [NT][Q][2] the pieces summed over the gM slots
  double* J;                 // [M] merit functional per state
  double* G;                 // [1]
  double* grad;              // [n_params]
  DevStatus* status;
  // grid-wide sweeps (N^2 > 4096): buffers of the iteration, [M*V] each
  int32_t gM;                // slots of gproj: M (one CTA per state), M * C * warps (cluster), 1 (grid)
  int32_t grid_blocks;       // blocks of the cooperative launch
  double2* zA;
  double2* zB;
  double2* lam;              // adjoint state
  double2* qf;               // recomputed forward state
  double* partials;          // [grid_blocks][LB_MAXQ][4] gradient pieces per block
  unsigned long long* gslots;  // [3][M] per-state |z_new - z| maxima, then [2][M] per-state |q| maxima
  GridBar* bar;
  double2* hist;             // [kRingOrder][M*V] first-iterate predictor history (grid and one-CTA sweeps)
  double2* Ginv;             // [V] 1/g, g = (1 + dt/2 D)/(1 - dt/2 D) the free step factor
  double2* hgp;              // [M*V] g^m per element of the ring hist's frame (m steps from its anchor)
  double2* hgm;              // [M*V] g^-m of the same
  double2* fgp;              // [M*V] the same for the ring histf
  double2* fgm;
  double2* histf;            // [kRingOrder][M*V] the forward predictor's history in a recompute (K > 0)
  int32_t pred_restart;      // forward predictor: -2 none, 0 never restarts, R > 0 restarts when j % R == 0
  int32_t pred_order;        // highest extrapolation order of the rotated predictor (1..kRingOrder)
  long long spin_limit;      // polls of a grid-barrier wait before it gives up (0: the kernels' default)
  uint32_t* hkl;             // [N (N + 1) / 2] the elements k <= l of the grid sweeps, k | l << 16, column by column
  int32_t herm;              // grid sweeps iterate k <= l only: every state and target is Hermitian
  int32_t diffit;            // grid sweeps: difference iterations in single precision allowed (Jacobi)
  float2* dfA;               // [M*V] grid sweeps: single-precision differences of successive iterates
  float2* dfB;
  float2* Dinvf;             // [V] grid sweeps: (I - dt/2 D)^-1 in single precision
  int32_t ff;                // grid sweeps: FP64 iterations apply O in single-precision pairs (lb_set_precision)
  int32_t pad2;
  float4* zsA;               // [M*V] the iterates zA / zB split into single-precision pairs (x_hi, x_lo, y_hi, y_lo)
  float4* zsB;
};

// one work item of a resident launch: (problem, state)
struct WorkItem {
  int32_t prob, state;
};

// ---- kernel launchers (lb_kernels.cu) --------------------------------------
namespace lbk {

constexpr int kMaxResidentV = 4096;  // states held in one CTA's shared memory
constexpr int kPredOrder = 7;        // extrapolation order of the cluster sweeps' first-iterate predictor
constexpr int kRingOrder = 10;       // ring slots (highest order) of the rotated first-iterate predictor
constexpr int kDefaultRingOrder = 8; // its default order (grid and one-CTA sweeps)

struct ResidentConfig {
  int threads;  // CTA size (multiple of 32, <= 512)
  int E;        // elements per thread (1, 2, 4, 8)
  int QT;       // E == 1: compile-time subsystem count of the per-thread plan (1..4), 0 = generic
  size_t smem;  // dynamic shared memory bytes
  bool gmres;   // kernels that can run GMRES (shared memory sized for its Krylov basis)
};

// uniformQ: every problem of the launch has Q = maxQ; kry_elems: complex
// values of the largest GMRES Krylov basis among them (0: no GMRES problem)
ResidentConfig resident_config(int maxV, int maxQ, int maxNcoef, int maxNj, int maxN, bool uniformQ,
                               size_t kry_elems = 0);
// GMRES cycle length m whose Krylov basis of m + 1 vectors fits one CTA's
// shared memory next to the resident sweep's buffers (0: below the minimum)
int gmres_krylov_dim(int V, int ncoef, int njcoef, int N, size_t smem_limit);

cudaError_t launch_tables(ProbDev* d_prob, const ProbDev& h_prob, cudaStream_t s);
cudaError_t launch_gate_targets(const ProbDev& h_prob, const double2* Vg, const int32_t* emap, const int32_t* efull,
                                int32_t Ne, cudaStream_t s);
cudaError_t launch_control_table(const ProbDev* d_prob, const ProbDev& h_prob, cudaStream_t s);
cudaError_t launch_forward_resident(const ProbDev* d_probs, const WorkItem* d_items, int n_items, int tape,
                                    const ResidentConfig& rc, cudaStream_t s);
cudaError_t launch_backward_resident(const ProbDev* d_probs, const WorkItem* d_items, int n_items,
                                     const ResidentConfig& rc, cudaStream_t s);
// objective (and gradient projection) for n_probs systems of the device array d_probs
cudaError_t launch_finalize(const ProbDev* d_probs, int n_probs, int max_param_warps, int with_grad, cudaStream_t s);
// copy G, gradients and status words of n_probs systems into contiguous arrays
cudaError_t launch_gather(const ProbDev* d_probs, int n_probs, const int64_t* grad_off, double* G_all,
                          double* grad_all, DevStatus* st_all, cudaStream_t s);
cudaError_t launch_apply(const ProbDev* d_prob, const ProbDev& h_prob, int adjoint, int64_t step, const double2* x,
                         double2* y, int n_vec, cudaStream_t s);
cudaError_t launch_propagate_resident(const ProbDev* d_prob, int adjoint, int64_t j0, int64_t j1, double2* x,
                                      int n_vec, const ResidentConfig& rc, cudaStream_t s);

// grid-wide cooperative sweeps for states too large for one CTA
constexpr int kGridThreads = 256;
constexpr int kMaxGridBlocks = 4096;
// largest cooperative grid of the sweep kernels on the current device
// blocks of the cooperative launch of the forward (backward = 0) or backward
// grid kernel in its FP64 (ff = 0) or paired-single form: all resident at once
int grid_blocks(int backward, int ff, size_t smem);
size_t grid_smem_bytes(int ncoef, int njcoef);
// mode 0: forward over [j0, j1) on P.qT (initialised from P.q0 when init_from_q0), checkpoints when tape;
// mode 1: forward over [j0, j1) in place on x; mode 2: adjoint steps j1-1..j0 in place on x
cudaError_t launch_sweep_grid(const ProbDev* d_prob, int mode, int init_from_q0, int tape, int64_t j0, int64_t j1,
                              double2* x, int nstates, int nblocks, size_t smem, int ff, cudaStream_t s);
cudaError_t launch_backward_grid(const ProbDev* d_prob, int nblocks, size_t smem, int ff, cudaStream_t s);

// cluster-split sweeps for small states: one cluster of C CTAs per state,
// 2Q lanes per element, or 4Q with the component split (Q <= 4,
// N^2 * lanes <= 1024)
struct ClusterConfig {
  int C;        // CTAs per cluster (0: not applicable)
  int QT;       // half pairs: subsystems plus Jaynes-Cummings pairs (compile-time kernel variant)
  int threads;  // threads per CTA
  size_t smem;  // dynamic shared memory per CTA
  bool cs;      // 4Q lanes per element (one per half and component) instead of 2Q
  bool pen;     // the running penalty (its own kernel instantiation)
};
ClusterConfig cluster_config(int V, int Q, int ncoef, int njcoef, int N, bool cs);
cudaError_t launch_forward_cluster(const ProbDev* d_prob, int M, int tape, const ClusterConfig& cc, cudaStream_t s);
cudaError_t launch_backward_cluster(const ProbDev* d_prob, int M, const ClusterConfig& cc, cudaStream_t s);
cudaError_t launch_propagate_cluster(const ProbDev* d_prob, int adjoint, int64_t j0, int64_t j1, double2* x, int n_vec,
                                     const ClusterConfig& cc, cudaStream_t s);
cudaError_t launch_objective_states(const ProbDev* d_prob, int M, cudaStream_t s);
// out[u] = qT[pmap[u] / 2], conjugate-transposed when pmap[u] is odd (u < Mu)
cudaError_t launch_expand_states(const double2* qT, const int32_t* pmap, int Mu, int N, double2* out, cudaStream_t s);

}  // namespace lbk
