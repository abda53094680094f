/*
 * lindblad_gb300.h -- C ABI of the GB300 (sm_103a) implicit-midpoint Lindblad
 * library: forward integration of the vectorised Lindblad master equation of
 * a composite qudit system, the objective, and its exact discrete-adjoint
 * gradient with respect to the B-spline control coefficients.
 *
 * The method (Guenther, Petersson, DuBois, "Quandary", arXiv:2110.10310):
 *   - model: Sec. II, master equation (mastereq), collapse operators
 *     L_1q = a_q/sqrt(T1), L_2q = a_q^+ a_q/sqrt(T2), cross-Kerr H_sys,
 *     rotating-frame control Hamiltonian H_c = sum_q d_q a_q + conj(d_q) a_q^+;
 *   - controls: eq. rotctrl, d_q(t) = sum_s S_s(t) sum_f alpha_q^{s,f} e^{i Omega_q^f t},
 *     quadratic B-splines with knot spacing T/(N_s - 2);
 *   - time stepping: Appendix A, eqs. mastereq_vectorized, IMR, linsystem_primal;
 *   - objective: Sec. III, eq. optimproblem with J_Frob or J_Tr (gamma1 = 0);
 *   - gradient: Appendix B, adjoint IMR, eq. linsystem_adjoint, eq. reducedgradient.
 *
 * Conventions shared by every call
 *   Units: frequencies are given as value/2pi in GHz, times in ns, T1/T2 in
 *     microseconds.  The library multiplies frequencies by 2pi.
 *   Ordering: subsystem 0 is the most significant digit of a basis index.
 *   Density matrices: M x N x N complex FP64, interleaved (re, im), COLUMN-major
 *     per matrix, i.e. element rho_i[k, l] is at double offset
 *     2 * (i * N * N + k + N * l).  This is vec(rho) of Appendix A (column
 *     stacking), so a state is exactly the vector q the method integrates.
 *   Control vector alpha: doubles laid out [q][f][s][re, im]; its length is
 *     2 * sum_q N_s * N_f(q).
 *   Return codes: LB_OK (0) or one of the LB_E* codes below.  On failure no
 *     output argument is written and lb_last_error() (thread-local) describes
 *     the cause; for LB_ENOTCONV and LB_ENAN it names the time step.
 *   Ownership: the library copies every host array it is given; the caller
 *     keeps ownership of its buffers.  Device memory is always provided by the
 *     caller (lb_workspace_bytes + lb_bind_workspace); the library never
 *     allocates device memory.
 *   Streams: every device call is asynchronous on the given CUDA stream
 *     (cudaStream_t passed as void*; NULL = legacy default stream) except where
 *     a host output is requested, in which case the call synchronises that
 *     stream before returning.
 *   Threads: a handle is not thread-safe; use one handle per host thread/stream.
 */
#ifndef LINDBLAD_GB300_H
#define LINDBLAD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define LB_OK 0
#define LB_EINVAL 1    /* invalid argument or call order */
#define LB_ENOMEM 2    /* workspace too small, or host allocation failed */
#define LB_ECUDA 3     /* a CUDA runtime call failed */
#define LB_ENOTCONV 4  /* the inner solve of some step did not converge within max_iter */
#define LB_ENAN 5      /* a state became NaN or Inf */

/* merit functionals, Sec. III */
#define LB_J_FROB 0 /* J = 1/2 ||rho_tar - rho||_F^2 */
#define LB_J_TR 1   /* J = 1 - Re Tr(rho_tar^+ rho) */
#define LB_J_NM 2   /* J = Tr(N_m rho), N_m = diag(|l - m|) over the full basis index l (lb_objective_set_measure) */

/* inner solvers for (I - dt/2 M) z = q, Appendix A (the paper solves it with
 * GMRES, Sec. IV); all converge to the same unique z:
 *   LB_SOLVER_JACOBI: z <- (I - dt/2 D)^-1 (q + dt/2 O z), D the diagonal of M
 *                     and O = M - D (the default; contraction ~ dt/2 |O|).
 *   LB_SOLVER_NEUMANN: z <- q + dt/2 M z (plain Neumann series).
 *   LB_SOLVER_GMRES: restarted GMRES(m) on the Jacobi-preconditioned system
 *                     (I - (I - dt/2 D)^-1 dt/2 O) z = (I - dt/2 D)^-1 q, for
 *                     steps where the fixed points converge slowly or diverge.
 *                     m <= 20 is the longest cycle whose Krylov basis fits one
 *                     CTA's shared memory beside the state (N^2 <= 1024 always
 *                     does); runs only in the one-CTA-per-state sweep, so
 *                     lb_bind_workspace fails with LB_EINVAL for grid or
 *                     cluster sweeps or a basis that does not fit.  Stops when
 *                     the 2-norm of the preconditioned residual (which bounds
 *                     the fixed-point increment of the rtol test) is below
 *                     rtol * max|q|; one iteration = one product with O.
 * LB_SOLVER_AUTO picks JACOBI (lb_autotune also times GMRES where it fits). */
#define LB_SOLVER_AUTO 0
#define LB_SOLVER_JACOBI 1
#define LB_SOLVER_NEUMANN 2
#define LB_SOLVER_GMRES 3

/* how the time loop is spread over the GPU:
 *   LB_SWEEP_RESIDENT: one CTA per state, the state in shared memory, the
 *                      whole time loop in one launch (N^2 <= 4096);
 *   LB_SWEEP_GRID:     one cooperative launch over all SMs and all states,
 *                      iterates in global memory, a grid barrier per inner
 *                      iteration (any N^2);
 *   LB_SWEEP_CLUSTER:  one thread-block cluster per state, each element's
 *                      work split over 2P or 4P lanes (P = Q + Jaynes-Cummings
 *                      pairs), the iterate replicated in every CTA's shared
 *                      memory (P <= 4, N^2 * 2P <= 1024);
 *                      for small states whose time loop is latency-bound;
 *   LB_SWEEP_AUTO:     GRID when N^2 > 4096 or when N^2 >= 1024 with fewer than
 *                      64 states (most SMs would idle); else CLUSTER when it
 *                      applies and all clusters fit on the GPU at once; else
 *                      RESIDENT. */
#define LB_SWEEP_AUTO 0
#define LB_SWEEP_RESIDENT 1
#define LB_SWEEP_GRID 2
#define LB_SWEEP_CLUSTER 3

#define LB_MAX_SUBSYSTEMS 8 /* Q <= 8 */
#define LB_MAX_LEVELS 64    /* n_q <= 64, and Q * max(4, ceil(log2 max n_q)) <= 32 */

typedef struct lb_system lb_system;
typedef struct lb_batch lb_batch;

/* System description (Sec. II).  All arrays are host memory and are copied. */
typedef struct lb_system_desc {
  int32_t Q;                   /* number of subsystems, 1..LB_MAX_SUBSYSTEMS */
  const int32_t* levels;       /* [Q] n_q >= 2 */
  const int32_t* essential;    /* [Q] essential levels per subsystem (gate objectives), NULL = all */
  const double* detuning_ghz;  /* [Q] (omega_q - omega_q^rot)/2pi */
  const double* selfkerr_ghz;  /* [Q] xi_q/2pi of -xi_q/2 a^+a^+aa, NULL = 0 */
  const double* crosskerr_ghz; /* [Q*Q] row-major; entry [p*Q+q], p<q, is xi_pq/2pi of -xi_pq n_p n_q; NULL = 0 */
  const double* t1_us;         /* [Q] decay time; <= 0 or inf switches L_1q off; NULL = all off */
  const double* t2_us;         /* [Q] dephasing time; <= 0 or inf switches L_2q off; NULL = all off */
  double T_ns;                 /* final time T > 0 */
  int64_t n_steps;             /* N_T >= 1; dt = T/N_T (uniform grid, Appendix A) */
} lb_system_desc;

/* Solver statistics of the last lb_forward / lb_gradient / lb_propagate.
 * Phases: 0 = forward sweep, 1 = recompute of checkpoint segments, 2 = adjoint
 * steps (which also evaluate the gradient pieces of eq. reducedgradient). */
typedef struct lb_stats {
  int64_t state_steps;      /* state-steps integrated, all phases */
  int64_t inner_iterations; /* fixed-point iterations summed over those state-steps */
  int32_t max_iterations;   /* largest iteration count of any single step */
  int32_t kernel_launches;  /* kernels launched by the call */
  int64_t phase_steps[3];   /* state-steps per phase */
  int64_t phase_iterations[3];
  float ms_forward;         /* device time of the forward-sweep kernel (lb_set_timing on, else 0) */
  float ms_backward;        /* device time of the backward-sweep kernel (recompute + adjoint) */
  int32_t sweep;            /* LB_SWEEP_* kind the call ran with */
  int32_t solver;           /* LB_SOLVER_* it ran with */
  int32_t ckpt_every;       /* checkpoint interval in effect (0 = every stage vector kept) */
  int32_t symmetry;         /* LB_SYM_HERMITIAN when the sweep iterated k <= l only */
  int32_t states_integrated; /* states the sweeps integrated (conjugate pairs count once, lb_set_pairing) */
  int32_t pad;
  int64_t phase_diff_iterations[3]; /* of phase_iterations: difference iterations in single precision
                                       (grid sweeps, lb_set_difference_iterations) */
} lb_stats;

/* ---- system ------------------------------------------------------------- */

/* Create a system from its description (Sec. II).  Errors: LB_EINVAL for
 * Q, levels, N_T or T out of range, or N = prod(n_q) > 2^15. */
int lb_system_create(const lb_system_desc* desc, lb_system** out);
void lb_system_destroy(lb_system* sys);

/* Control parameterisation, eq. rotctrl: n_splines >= 3 quadratic B-splines
 * per subsystem and n_carriers[q] >= 1 carrier frequencies for subsystem q;
 * carrier_ghz holds Omega_q^f/2pi for all q, f, concatenated in q-major order.
 * Resets alpha to zero. */
int lb_controls_define(lb_system* sys, int32_t n_splines, const int32_t* n_carriers, const double* carrier_ghz);

/* Interval [0, T_c] the B-splines of eq. rotctrl span (knot spacing
 * T_c/(N_s - 2)): T_c = T_ns, or the system's final time T for T_ns = 0 (the
 * default).  A system that integrates the first N_T steps of a longer
 * horizon (its T = N_T dt) keeps that horizon's controls by setting T_c to
 * the longer horizon.  LB_EINVAL for a negative or non-finite T_ns; call
 * before lb_bind_workspace. */
int lb_controls_set_horizon(lb_system* sys, double T_ns);

/* Set the control vector alpha (host, length n = 2 sum_q N_s N_f(q); layout
 * [q][f][s][re, im], GHz).  If a workspace is bound, the copy to the device
 * is issued on the bound stream before returning. */
int lb_controls_set(lb_system* sys, const double* alpha, int64_t n);

/* Initial states rho_i(0), i < M (host, M x N x N complex, column-major) and
 * weights beta_i (host, [M], NULL = all 1).  The objective divides by M
 * (eq. optimproblem).  M may only change while no workspace is bound.  If a
 * workspace is bound, the copy to the device is issued before returning. */
int lb_states_set(lb_system* sys, int32_t M, const double* rho0, const double* weights);

/* Objective with explicit targets rho_i^tar (host, M x N x N complex,
 * column-major; call after lb_states_set) and Tikhonov weight gamma2 >= 0. */
int lb_objective_set(lb_system* sys, int32_t kind, const double* targets, double gamma2);

/* Gate objective (Sec. III-C): rho_i^tar = V rho_i(0) V^+ with V (host,
 * Ne x Ne complex, interleaved, column-major, Ne = prod essential levels)
 * lifted to the full space by the isometry that maps essential digits to the
 * same digits of the full space (zero on guard levels).  Uses the states set
 * by lb_states_set; the targets are computed on the device. */
int lb_objective_set_gate(lb_system* sys, int32_t kind, const double* V, double gamma2);

/* Inner solver and checkpointing.  rtol: stop when
 * max|z_new - z| <= rtol * max|q| * f_j (componentwise, per state), where for
 * the Jacobi iteration f_j = (1 - rho_j)/rho_j with rho_j < 1/2 an upper bound
 * of the infinity norm of its iteration matrix at step j (then
 * max|z - z*| <= rtol * max|q| for the returned z), and f_j = 1 otherwise
 * (rho_j >= 1/2, or the Neumann iteration); max_iter caps the
 * iterations of one step (LB_ENOTCONV beyond); ckpt_every = K >= 1 stores the
 * forward state every K steps and recomputes each K-step segment in the
 * backward sweep; K = 0 stores every stage vector z^j instead (no recompute);
 * K = LB_CKPT_AUTO keeps every stage vector when that tape takes at most
 * 8 GiB (M * N_T * N^2 * 16 bytes) and checkpoints every 100 steps otherwise.
 * Defaults: LB_SOLVER_AUTO, 1e-15, 200, 100.  Call before lb_workspace_bytes. */
#define LB_CKPT_AUTO (-1)
int lb_solver_set(lb_system* sys, int32_t method, double rtol, int32_t max_iter, int32_t ckpt_every);

/* Merit functional J_Nm (Sec. III-B, eq. Jmeasure) for every state:
 * J = Tr(N_m rho(T)) with the observable N_m = diag(|l - m|), l = 0..N-1 the
 * full basis index, which vanishes only at rho = |m><m| (unconditional
 * preparation of |m><m|, e.g. ground-state reset m = 0, usually from the
 * single ensemble state 1/N^2 sum_kj B^kj).  Terminal adjoint condition
 * beta_i/M vec(N_m).  LB_EINVAL for m outside 0..N-1 or a bad gamma2; call
 * after lb_states_set. */
int lb_objective_set_measure(lb_system* sys, int32_t m, double gamma2);

/* Running penalty of eq. optimproblem (Sec. III):
 *   G += gamma1/M sum_i beta_i sum_{j=0}^{N_T-1} dt beta(t_j) J(rho_i^tar, rho_i(t_j)),
 *   beta(t) = exp(-((t - T)/a)^2)/a,
 * the time integral by the left rectangle rule, weighted per state like the
 * final-time term; its derivative enters the adjoint sweep as the source
 * gamma1 beta_i/M dt beta(t_j) g(q^j) at qhat^j (Appendix B).  gamma1 >= 0
 * (0 = off, the default), a_ns > 0.  Runs in every sweep; LB_SWEEP_AUTO
 * keeps states with N^2 <= 4096 on the one-CTA-per-state or cluster sweeps.
 * The grid sweep sums each step's merit per block over the states its
 * contiguous share of the elements covers, so lb_bind_workspace refuses it
 * (LB_EINVAL) when a block's share spans more than 4 states (very many small
 * states).  Call before lb_workspace_bytes. */
int lb_objective_set_penalty(lb_system* sys, double gamma1, double a_ns);

/* Conjugate pairs of initial states (Sec. III-B: the basis |k><j| of a gate
 * objective holds |k><j| and |j><k| = (|k><j|)^+).  Lindblad's equation and
 * the implicit midpoint step commute with the conjugate transpose, so with
 * on = 1 (the default) a state that is exactly (entry by entry) the
 * conjugate transpose of an earlier one, and whose explicit target is that
 * earlier target's conjugate transpose (gate and J_Nm targets follow), is not
 * integrated: its final state is the conjugate transpose of its partner's,
 * its merit equals the partner's (J_Frob, J_Tr and J_Nm are invariant), and
 * so does its share of the gradient (eq. reducedgradient), so the partner is
 * integrated once with the sum of both weights.  lb_forward still returns all
 * M final states; lb_stats.states_integrated and the state-steps count the
 * integrated ones.  With a workspace bound, new states or targets must pair
 * the same way (LB_EINVAL otherwise).  on = 0 integrates every state.  Call
 * before lb_workspace_bytes. */
int lb_set_pairing(lb_system* sys, int32_t on);

/* Choose the sweep kind (LB_SWEEP_*); call before lb_workspace_bytes. */
int lb_set_sweep(lb_system* sys, int32_t sweep);

/* First iterate of the inner solves (Appendix A, eq. linsystem_primal; the
 * paper does not say how its Krylov solve is started).  Every solve starts
 * from (I - dt/2 D)^-1 (q^j + c~), c~ the extrapolation of the off-diagonal
 * corrections c = (I - dt/2 D) z - q of the previous steps by the polynomial
 * through them; the grid and one-CTA sweeps extrapolate each element in the
 * frame of its own free evolution, g = 2 (I - dt/2 D)^-1 - 1 per step, up to
 * `order` (1..10; 0 = the default, 8), the cluster sweep without the frame up
 * to order 7.  The adjoint sweep always predicts.  `restart` says when the
 * forward predictor forgets its history (it then rebuilds it over the next
 * steps):
 *   LB_PRED_AUTO (default): every K steps with checkpoints (K > 0), never
 *     with the full stage tape (K = 0);
 *   R > 0: at every step j with j % R == 0; with K > 0, R must divide K;
 *   0: never; only with K = 0 (lb_bind_workspace fails with LB_EINVAL else);
 *   LB_PRED_NONE: no forward predictor, the first iterate is
 *     (I - dt/2 D)^-1 q^j.
 * A checkpoint is always a restart point, so a recompute of a checkpoint
 * segment repeats the forward sweep's iterates bit for bit: for a given
 * restart period R the gradient with checkpoints every K (R | K) is bitwise
 * that of the full tape (K = 0), and results for different R agree to
 * rounding.  The cluster sweep (LB_SWEEP_CLUSTER) predicts its forward
 * solves only with K = 0.  Call before lb_workspace_bytes. */
#define LB_PRED_AUTO (-1)
#define LB_PRED_NONE (-2)
int lb_set_predictor(lb_system* sys, int32_t restart, int32_t order);

/* The forward predictor's restart period in effect (LB_PRED_NONE, 0 or R;
 * see lb_set_predictor) and its order (which lb_autotune may have chosen).
 * Either output pointer may be NULL. */
int lb_get_predictor(const lb_system* sys, int32_t* restart, int32_t* order);

/* Bound of the grid sweeps' barrier waits (failure detection; the paper has
 * no counterpart).  Each block polls the grid barrier at most `polls` times
 * (about 64 ns apart) before it gives up; a wait that gives up makes every
 * block of the launch return, and the call reports LB_ECUDA with the time
 * step ("a grid barrier wait gave up at time step j").  The handle stays
 * usable: the next call clears the barrier.  0 restores the default
 * (2^26 polls, seconds).  May be called at any time; with a workspace bound
 * the new bound is uploaded on the bind stream, which is synchronised. */
int lb_set_wait_limit(lb_system* sys, int64_t polls);

/* Single-precision difference iterations of the grid sweeps' Jacobi solves
 * (on = 1, the default; 0 = every inner iteration in FP64).  The implicit
 * midpoint step (I - dt/2 M) z = q (Appendix A, eqs. IMR, linsystem_primal) is solved by
 * z_{k+1} = (I - dt/2 D)^-1 (q + c(z_k)), c(z) = (dt/2) O z, O the
 * off-diagonal part of M.  Once every state's last change
 * d_k = z_k - z_{k-1} is below 2^-32 max|q| (and max|q| >= 2^-50), the next
 * iteration computes c(z_k) - c(z_{k-1}) = (dt/2) O d_k and
 * z_{k+1} - z_k = (I - dt/2 D)^-1 (dt/2) O d_k in single precision from d_k
 * rounded to single precision, and adds them to the FP64 correction and
 * iterate.  Their rounding errors are below 2^-24 of terms that are already
 * below 2^-32 of the state, under the FP64 rounding of z, and the stopping
 * rule (rtol) is unchanged; the first iteration of every step is FP64.  The
 * one-CTA and cluster sweeps, GMRES and the Neumann series ignore the
 * switch.  lb_stats.phase_diff_iterations counts these iterations.  May be
 * called at any time; with a workspace bound the switch is uploaded on the
 * bind stream, which is synchronised. */
int lb_set_difference_iterations(lb_system* sys, int32_t on);

/* Arithmetic of the grid sweeps' FP64 inner iterations (the first of every
 * step and any before the difference iterations take over).
 *   LB_PREC_F64 (default): the off-diagonal apply c = (dt/2) O z in FP64.
 *   LB_PREC_F32X2: the apply in pairs of single-precision numbers (hi + lo,
 *     about 48 significant bits): every iterate is also stored split into
 *     such pairs, each product of a coefficient and a neighbour is formed
 *     with its exact rounding error and the sums carry theirs (two-sum), so
 *     c is within about 2^-48 of the sum of the magnitudes of its terms,
 *     i.e. within about 2^-48 rho |z| where rho < 1 is the Jacobi
 *     contraction bound: a few FP64 roundings of z, under the solver's
 *     tolerance (the off-diagonal part c of the implicit midpoint step,
 *     Appendix A, is at most about rho |z|).  The FP64 pipe, which runs at
 *     1/64 of the single-precision rate on this GPU, then only forms
 *     z = (I - dt/2 D)^-1 (q + c).  States, the right-hand side, the diagonal, the objective,
 *     the gradient pieces and the stopping rule stay FP64.  Systems with
 *     Jaynes-Cummings couplings keep LB_PREC_F64.  Call before
 *     lb_workspace_bytes (the split iterates take 32 bytes per element and
 *     state). */
#define LB_PREC_F64 0
#define LB_PREC_F32X2 1
int lb_set_precision(lb_system* sys, int32_t precision);

/* Jaynes-Cummings coupling of the system Hamiltonian (Sec. II):
 *   sum_{p<q} g_pq (e^{i eta_pq t} a_p^+ a_q + e^{-i eta_pq t} a_p a_q^+),
 *   eta_pq = omega_p^rot - omega_q^rot,
 * the general rotating-frame form with time-dependent factors.  jc_ghz:
 * Q x Q row-major g_pq/2pi in GHz, entries p < q used (0 = no coupling);
 * rot_ghz: Q rotating-frame frequencies omega_q^rot/2pi in GHz (nullable: all
 * equal, eta = 0).  Copied.  Call before lb_workspace_bytes; each pair adds
 * two halves to a cluster sweep's lane plan (see LB_SWEEP_CLUSTER). */
int lb_system_set_coupling(lb_system* sys, const double* jc_ghz, const double* rot_ghz);

/* Hermitian symmetry (Sec. III-B: density matrices, and Lindblad's equation
 * preserves Hermiticity).  It applies when every initial state set by
 * lb_states_set and every explicit target is Hermitian to rounding (each
 * entry within 64 eps max|entry| of the conjugate of its transposed entry;
 * the k <= l entries are then used for both), gate targets V rho V^+ being
 * Hermitian with their states.  A sweep under it iterates only the elements
 * k <= l of every state and writes the conjugate into (l, k) (the grid
 * sweeps keep them packed): about half the work.  The adjoint states are
 * then Hermitian too and the gradient pieces of the mirrored elements are
 * formed from those of (k, l).
 *   LB_SYM_HERMITIAN: every sweep kind -- grid-wide, one CTA per state
 *     (fixed points and GMRES, whose inner products are then real) and
 *     cluster.
 *   LB_SYM_AUTO (the default): the grid and one-CTA sweeps, not the cluster
 *     sweep, whose steps are bound by latency rather than by the number of
 *     elements.
 *   LB_SYM_NONE: every element is always iterated.
 * May be called at any time; applies from the next call. */
#define LB_SYM_NONE 0
#define LB_SYM_HERMITIAN 1
#define LB_SYM_AUTO 2
int lb_set_symmetry(lb_system* sys, int32_t symmetry);

/* ---- device workspace ---------------------------------------------------- */

/* Bytes of device memory the system needs (depends on N, M, N_T, Q, the
 * control layout and ckpt_every).  When the grid-wide sweep runs under the
 * Hermitian symmetry (Hermitian states and targets, LB_SYM_AUTO or
 * LB_SYM_HERMITIAN), its checkpoint and segment tapes are sized for the
 * k <= l entries of each state, N (N + 1) / 2 instead of N^2; a workspace
 * bound so refuses later calls (LB_EINVAL, "packed tapes") while the states
 * or targets set since are not Hermitian or the symmetry is switched off,
 * until they are Hermitian again or a new workspace is bound. */
int lb_workspace_bytes(const lb_system* sys, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned, >= lb_workspace_bytes)
 * and upload every table, state, target and the controls on `stream`.
 * The memory must stay valid until the system is destroyed or rebound. */
int lb_bind_workspace(lb_system* sys, void* dev_workspace, size_t bytes, void* stream);

/* ---- the method ---------------------------------------------------------- */

/* Forward sweep over the whole horizon for all M states, then the objective
 * G (eq. optimproblem).  G_out (host, nullable) receives G; rhoT_dev_out
 * (device, nullable, M x N x N complex) receives rho_i(T). */
int lb_forward(lb_system* sys, void* stream, double* G_out, void* rhoT_dev_out);

/* Forward sweep with checkpoints, then the discrete adjoint sweep (Appendix B)
 * with the reduced gradient.  G_out (host, nullable) receives G; grad_out
 * (host, nullable, length of alpha) receives dG/dalpha. */
int lb_gradient(lb_system* sys, void* stream, double* G_out, double* grad_out);

/* Minimise G(alpha) by L-BFGS (Sec. III and Appendix B: the paper updates the
 * control vector with L-BFGS steps built from the adjoint gradient; two-loop
 * recursion of Nocedal & Wright, Numerical Optimization, Algorithm 7.4).
 * Starts from the controls set last (lb_controls_set) and leaves the final
 * iterate set; every function value and gradient is one lb_gradient on
 * `stream`.  Direction -H_k g with H_k^0 = (s^T y / y^T y) I of the newest of
 * at most `memory` pairs (a pair is kept only when s^T y > 1e-10 |s| |y|);
 * with no pair, -g scaled to max-norm `step0`.  Backtracking from the unit
 * step, halving until G(x + t d) <= G(x) + 1e-4 t g^T d (at most 30 trials,
 * after which the run stops at the current iterate).  Stops when
 * max|grad| <= gtol or after max_iter accepted steps.
 * Outputs (host, nullable): G_out the final G; alpha_out the final alpha
 * (length of alpha); iters_out the accepted steps; evals_out the gradient
 * evaluations; history [max_iter + 1][2] receives (G, max|grad|) of the start
 * and of every accepted iterate.  LB_EINVAL for memory < 1, max_iter < 0,
 * gtol < 0 or step0 <= 0; errors of a gradient evaluation are returned as
 * they are (the controls then hold the iterate that failed). */
int lb_optimize(lb_system* sys, void* stream, int32_t max_iter, int32_t memory, double gtol, double step0,
                double* G_out, double* alpha_out, int32_t* iters_out, int32_t* evals_out, double* history);

/* Device-resident variant of lb_gradient: G and the gradient are written to
 * device memory (G_dev: 1 double, grad_dev: length of alpha) and the call
 * does not synchronise; errors of the device sweep are reported by the next
 * synchronising call. */
int lb_gradient_async(lb_system* sys, void* stream, void* G_dev, void* grad_dev);

/* Advance n_vec device vectors x (n_vec x N x N complex, column-major) from
 * step j0 to step j1 (0 <= j0 <= j1 <= N_T) with the implicit midpoint rule
 * (adjoint = 0), or apply the adjoint steps j1-1 down to j0 to them
 * (adjoint = 1: (I - dt/2 M^+) zhat = x, x <- 2 zhat - x).  In place.
 * With grid sweeps n_vec <= M (the iteration buffers hold M states). */
int lb_propagate(lb_system* sys, void* stream, int32_t adjoint, int64_t j0, int64_t j1, void* x_dev, int32_t n_vec);

/* y = M^{j+1/2} x (adjoint = 0) or y = (M^{j+1/2})^+ x (adjoint = 1) for
 * n_vec device vectors (Appendix A, eq. mastereq_vectorized), with
 * M^{j+1/2} = M(t_j + dt/2); x and y must not overlap. */
int lb_apply(lb_system* sys, void* stream, int32_t adjoint, int64_t step, const void* x_dev, void* y_dev,
             int32_t n_vec);

/* Statistics of the last forward / gradient / propagate call. */
int lb_get_stats(lb_system* sys, lb_stats* out);

/* Autotuner: time `probe_steps` forward steps (from the initial states, on
 * the device; results discarded) of every candidate compatible with the bound
 * workspace -- sweep kind (one CTA per state with 1, 2, 4 or 8 elements per
 * thread, cluster-split when it applies; grid when the workspace was bound
 * for grid sweeps) x inner solver (Jacobi, Neumann, and GMRES for one CTA
 * per state where its Krylov basis fits) -- and keep the fastest
 * candidate whose inner solve converges for later calls.  Grid sweeps with a
 * forward predictor then time the forward sweep with the predictor over the
 * first max(probe_steps, 30) steps for the orders 6..10 and keep the fastest
 * (lb_get_predictor reports it).  Synchronises
 * `stream`.  choice_out (nullable, [3]) receives the chosen LB_SWEEP_*,
 * LB_SOLVER_* and the threads per CTA (resident), CTAs per cluster (cluster)
 * or blocks (grid).  LB_ENOTCONV when no candidate converges. */
int lb_autotune(lb_system* sys, void* stream, int32_t probe_steps, int32_t* choice_out);

/* on != 0: record CUDA events around the sweep kernels on the launching
 * stream and report their device time in lb_stats (ms_forward, ms_backward)
 * after the next synchronising call. */
int lb_set_timing(lb_system* sys, int32_t on);

/* ---- gradient without device allocation ----------------------------------- */

/* Size of the device array behind lb_gradient_static: 64 MiB, held on every
 * GPU that loads this library until the process exits. */
#define LB_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)

/* Same result as lb_gradient, for callers that cannot allocate device memory
 * (code running inside a host callback, a framework that owns all device
 * memory, a control loop that must not touch the allocator).  The paper has no
 * counterpart: this is a deployment variant of lb_gradient.
 *
 * The handle carries the inputs (controls, states, objective, solver, set by
 * the calls above) and must NOT have a workspace bound; G_out and grad_out
 * are host outputs as in lb_gradient.  Every table, checkpoint, tape and
 * partial result of the call lives in one file-scope device array of
 * LB_STATIC_SCRATCH_BYTES; nothing is allocated on the device, by the library
 * or by anything it calls.  A problem whose lb_workspace_bytes exceeds
 * LB_STATIC_SCRATCH_BYTES is rejected with LB_ENOMEM.
 *
 * The call always runs one CTA per state: a handle given
 * lb_set_sweep(LB_SWEEP_CLUSTER) (or a grid-sized problem) is refused with
 * LB_EINVAL.  Each call looks the array's device address up with the current
 * device current (the first call on a device also loads the module there:
 * make it before any stream capture; during a capture the address found by
 * the last call outside one is used).  All calls share the one array: every
 * call clears the part of it the problem uses and uploads all of the
 * handle's inputs again (states, targets, tables, controls), so each call
 * pays that host-to-device copy, and calls that overlap on the GPU (other
 * streams, other host threads, another handle) race with each other and
 * must be serialised by the caller.  The call synchronises `stream` before it
 * returns, on error returns too once device work was queued, and leaves the
 * handle unbound. */
int lb_gradient_static(lb_system* sys, void* stream, double* G_out, double* grad_out);

/* ---- batches of independent problems ------------------------------------- */

/* A batch of n >= 1 independent systems, each already bound to its own
 * workspace, advanced together in one persistent launch per sweep (the
 * paper's first level of parallelism, Sec. V).  The batch needs a small
 * workspace of its own. */
int lb_batch_create(lb_system* const* systems, int32_t n, lb_batch** out);
void lb_batch_destroy(lb_batch* batch);
int lb_batch_workspace_bytes(const lb_batch* batch, size_t* bytes);
int lb_batch_bind_workspace(lb_batch* batch, void* dev_workspace, size_t bytes, void* stream);

/* G_out (host, nullable, [n]) per system; grad_out (host, nullable) the
 * gradients of all systems concatenated in batch order. */
int lb_batch_forward(lb_batch* batch, void* stream, double* G_out);
int lb_batch_gradient(lb_batch* batch, void* stream, double* G_out, double* grad_out);

/* Capture the device work of lb_batch_forward (mode 0) or lb_batch_gradient
 * (mode 1) into a CUDA graph; later calls of that mode replay the graph.
 * mode -1 drops the graphs. */
int lb_batch_capture_graph(lb_batch* batch, void* stream, int32_t mode);

/* Statistics summed over the batch's last call. */
int lb_batch_get_stats(lb_batch* batch, lb_stats* out);

/* ---- diagnostics --------------------------------------------------------- */

/* Description of the last error of the calling thread ("" if none). */
const char* lb_last_error(void);

/* Library version string. */
const char* lb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LINDBLAD_GB300_H */
