// Small kernels of the implicit-midpoint Lindblad path: time-independent
// tables, gate targets, the control table and stopping factors, objective
// and gradient projection, the batch gather, and the Lindblad apply.

#include "lb_device.cuh"

namespace lbk {

namespace {

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
    if (P.Dinvf) P.Dinvf[tid] = make_float2((float)(ar / den), (float)(-ai / den));
    if (P.Ginv) {
      // 1/g = (1 - dt/2 D)/(1 + dt/2 D), g the element's free step factor
      const double br = 1.0 + hh * D.x, bi = hh * D.y;
      const double bd = br * br + bi * bi;
      P.Ginv[tid] = make_double2((ar * br + ai * bi) / bd, (ai * br - ar * bi) / bd);
    }
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
  const double dtau = P.Tc / (P.Ns - 2);
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
  const double dtau = P.Tc / (P.Ns - 2);
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


// The final state of every given state (lb_forward): its integrated state,
// or for the second state of a conjugate pair the conjugate transpose of its
// partner's (Lindblad's equation and the implicit midpoint step commute with
// the conjugate transpose).
__global__ void k_expand_states(const double2* __restrict__ qT, const int32_t* __restrict__ pmap, int Mu, int N,
                                double2* __restrict__ out) {
  const size_t V = (size_t)N * N;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)Mu * V) return;
  const int u = (int)(t / V);
  const int v = (int)(t - (size_t)u * V);
  const int e = pmap[u] >> 1;
  if (pmap[u] & 1) {
    const int k = v % N, l = v / N;
    const double2 x = qT[(size_t)e * V + l + (size_t)N * k];
    out[t] = make_double2(x.x, -x.y);
  } else {
    out[t] = qT[(size_t)e * V + v];
  }
}
}  // namespace

// ---------------------------------------------------------------------------
// launchers

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

cudaError_t launch_expand_states(const double2* qT, const int32_t* pmap, int Mu, int N, double2* out, cudaStream_t s) {
  const size_t n = (size_t)Mu * N * N;
  k_expand_states<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(qT, pmap, Mu, N, out);
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

}  // namespace lbk
