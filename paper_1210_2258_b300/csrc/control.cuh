// Scalar decisions of the methods, taken on the device by the block that finishes a row pass last
// (see arrive_last), so an iteration never waits on the host and needs no controller launch.
// Every function is called by all threads of that block; thread 0 takes the decisions.
//   ctrl_sgp_begin         after K1: k <- k+1 once the pending update is applied, J_0 (Eq. KL),
//                          min-error rule, completion of a decided stop
//   ctrl_sgp_alpha         after K3: step 1 of Alg. 1, scaled BB values (Eq. BB1, BB2), the
//                          safeguards, the alternation of Eq. (alphadef) with the M_alpha window
//                          and tau, warm-up rule
//   ctrl_sgp_lambda        after K6: step 5 of Alg. 1, first lambda in {1} ({1, theta} after one
//                          backtrack, {1, .., theta^3} after more) with
//                          J(f + lambda d) <= J(f) + beta lambda grad'd; stop rules of Sect. 3.3
//   ctrl_sgp_lambda_extra  after K7: the remaining powers up to theta^30 when needed
//   ctrl_rl                after the RL ratio pass: Richardson-Lucy bookkeeping (J, trace, stops)
#pragma once
#include <math.h>
#include "reduce.cuh"
#include "state.cuh"

namespace sgp {

__device__ inline void trace_push(double* trace, CtrlState* c, double k, double J, double alpha,
                                  double lam, int bt, int branch, double gTd) {
  if (trace && c->trace_n < c->trace_cap) {
    double* r = trace + size_t(c->trace_n) * kTraceStride;
    r[0] = k; r[1] = J; r[2] = 2.0 * J * c->inv_pS; r[3] = alpha; r[4] = lam;
    r[5] = bt; r[6] = branch; r[7] = gTd;
  }
  c->trace_n += 1;
}

// Step 1 of Alg. 1 for k >= 1 (V = double, or float for the plain-FP32 variant).
template <class V>
__device__ inline double bb_alpha(CtrlState* c, V n1, V d1, V n2, V d2, int k) {
  const V amin = V(c->alpha_min), amax = V(c->alpha_max), aprev = V(c->alpha);
  // both quotients before either is used, so that the two (long-latency) divisions overlap; a
  // quotient whose guard fails is not used
  const V q1 = n1 / d1, q2 = n2 / d2;
  const V a1 = d1 <= V(0) ? fmin(V(10) * aprev, amax) : fmin(amax, fmax(amin, q1));
  const V a2 = n2 <= V(0) ? fmin(V(10) * aprev, amax) : fmin(amax, fmax(amin, q2));
  // window of the last M_alpha values of alpha^(2), Eq. (alphadef)
  if (c->hist_n < c->M_alpha) c->hist[c->hist_n++] = double(a2);
  else {
    for (int i = 1; i < c->M_alpha; ++i) c->hist[i - 1] = c->hist[i];
    c->hist[c->M_alpha - 1] = double(a2);
  }
  V wmin = V(c->hist[0]);
  for (int i = 1; i < c->hist_n; ++i) wmin = fmin(wmin, V(c->hist[i]));
  V alpha;
  if (k <= c->warmup) { alpha = wmin; c->branch = 2; }
  else if (a2 <= V(c->tau) * a1) { alpha = wmin; c->tau *= 0.9; c->branch = 2; }   // a2 / a1 <= tau, a1 > 0
  else { alpha = a1; c->tau *= 1.1; c->branch = 1; }
  return double(alpha);
}

// The controller's working copy of the state: every thread loads up to kCtrlPer 8-byte words of it
// (in flight while the partial sums are read), thread 0 decides on the shared copy, the block
// writes it back.  Blocks have at least 32 threads.
constexpr int kCtrlWords = int(sizeof(CtrlState) / 8);
constexpr int kCtrlPer = 4;
static_assert(sizeof(CtrlState) % 8 == 0 && kCtrlWords <= 32 * kCtrlPer,
              "controller state must fit kCtrlPer words per thread of a 32-thread block");
struct CtrlCopy {
  unsigned long long w[kCtrlPer];
  __device__ __forceinline__ explicit CtrlCopy(const CtrlState* c) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(c);
#pragma unroll
    for (int k = 0; k < kCtrlPer; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      w[k] = i < kCtrlWords ? __ldcg(src + i) : 0ull;
    }
  }
  __device__ __forceinline__ void to_shared(CtrlState& s) const {
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s);
#pragma unroll
    for (int k = 0; k < kCtrlPer; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < kCtrlWords) dst[i] = w[k];
    }
    __syncthreads();
  }
  __device__ __forceinline__ static void write_back(const CtrlState& s, CtrlState* c) {
    __syncthreads();
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&s);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(c);
    for (int i = threadIdx.x; i < kCtrlWords; i += blockDim.x) dst[i] = src[i];
  }
};

template <bool FP64>
__device__ void sgp_begin_decide(CtrlState* c, const double (&kl)[2]) {
  const int done = c->done;
  if (!c->fresh) {
    c->k += 1;
    c->fresh = 1;
    c->f_pending = f_update_in_k1(c, done) ? 0 : 1;
    c->R = c->R_pred;                 // the Tikhonov term moves with the step (exact in lambda)
  }
  if (done == 1) { c->done = 2; c->J = c->J_pred; return; }
  if (!isfinite(kl[0])) {   // stop at the last stored iterate (a pending f^(k) is not formed)
    c->status = 8; c->done = 2;
    if (c->f_pending) { c->k -= 1; c->f_pending = 0; }
    return;
  }
  c->J = kl[0];
  if (c->stop_kind == STOP_MIN_ERROR && c->ftrue_norm2 > 0.0) {
    const double rho = sqrt(kl[1] / c->ftrue_norm2);
    c->rho = rho;
    if (c->k >= 1 && rho > c->rho_prev) { c->done = 2; c->result_prev = 1; return; }
    c->rho_prev = rho;
  }
}
// The per-iteration controllers (the three of SGP here, ctrl_rl below) run for real in the block
// that arrives last; with `dry` they write nothing to global memory and no trace record.  A
// controller's instructions run once per pass, in one block, after ~20 us in which the pass has
// streamed tens of MB through L2: fetched cold, they cost that block 1-2 us of the ~40 000-cycle
// pass.  So in the one-wave passes over rows of 2048 the blocks that arrive before the last one
// (which have nothing else to do) run the controller dry first, which brings its code into L2 and
// into the instruction caches of their SMs.  They call the one non-inlined copy (the *_nl ones) that
// the last block calls, so the dry runs warm the code that the real run executes.  Elsewhere the
// controller runs in the last block only: inlined at the other widths (64 registers per thread,
// where a call's saved registers would spill), and without dry runs in passes of several waves (a
// dry run would hold a slot that a waiting block needs) or of fewer blocks than SMs (the arrivals
// do not spread enough for the dry runs to end first); ImgDesc::dry_row / dry_rv say which.
// (with done == 1 the KL partials were not written by this pass: the sums are not used)
template <bool FP64>
__device__ __forceinline__ void ctrl_sgp_begin(const ImgDesc& d, bool dry) {
  __shared__ CtrlState s;
  const CtrlCopy cp(d.ctrl);
  double kl[2];
  ctrl_sum<2, FP64>(d, SLOT_KL, kl, true);
  cp.to_shared(s);
  if (threadIdx.x == 0) sgp_begin_decide<FP64>(&s, kl);
  if (!dry) CtrlCopy::write_back(s, d.ctrl);
  else __syncthreads();
}
template <bool FP64>
__device__ __noinline__ void ctrl_sgp_begin_nl(const ImgDesc& d, bool dry) { ctrl_sgp_begin<FP64>(d, dry); }

template <bool FP64>
__device__ void sgp_alpha_decide(CtrlState* c, const double (&bb)[4]) {
  double alpha;
  if (c->k == 0) {
    alpha = c->alpha0;
    c->branch = 0;
  } else if (FP64) {
    alpha = bb_alpha<double>(c, bb[0], bb[1], bb[2], bb[3], c->k);
  } else {
    alpha = bb_alpha<float>(c, float(bb[0]), float(bb[1]), float(bb[2]), float(bb[3]), c->k);
  }
  c->alpha = alpha;
  c->f_pending = 0;   // K3 has stored f^(k)
}
template <bool FP64>
__device__ __forceinline__ void ctrl_sgp_alpha(const ImgDesc& d, bool dry) {
  __shared__ CtrlState s;
  const CtrlCopy cp(d.ctrl);
  double bb[4];
  ctrl_sum<4, FP64>(d, SLOT_BB, bb, false);
  cp.to_shared(s);
  if (threadIdx.x == 0) sgp_alpha_decide<FP64>(&s, bb);
  if (!dry) CtrlCopy::write_back(s, d.ctrl);
  else __syncthreads();
}
template <bool FP64>
__device__ __noinline__ void ctrl_sgp_alpha_nl(const ImgDesc& d, bool dry) { ctrl_sgp_alpha<FP64>(d, dry); }

// Change of the Tikhonov term beta/2 ||f||^2 along the step: R(f + lam d) - R(f) =
// beta (lam f'd + lam^2/2 d'd), exact in lam (0 without regularisation)
__device__ __forceinline__ double reg_delta(const CtrlState* c, double lam) {
  return c->reg_beta > 0.0 ? c->reg_beta * (lam * c->reg_fd + 0.5 * lam * lam * c->reg_dd) : 0.0;
}

__device__ inline void sgp_accept(double* trace, CtrlState* c, int nb, double lam, double dJ) {
  c->lambda = lam;
  c->backtracks = nb;
  c->dJ = dJ;
  c->J_pred = c->J + dJ;
  c->R_pred = c->R + reg_delta(c, lam);
  c->fresh = 0;                       // f^(k+1) = f^(k) + lambda d is applied by the next K1
  c->need_more = 0;
  c->arm_nl = nb == 0 ? 1 : (nb == 1 ? 2 : kArmMain);
  const int kn = c->k + 1;
  trace_push(trace, c, kn, c->J_pred, c->alpha, lam, nb, c->branch, c->gTd);
  bool rule = false;                  // the stop rule itself fired (not only the iteration cap)
  // Eq. (convergence) on the objective J_0 + R (R = 0 without regularisation)
  if (c->stop_kind == STOP_CONVERGENCE &&
      fabs((c->J_pred + c->R_pred) - (c->J + c->R)) <= c->tol * (c->J + c->R)) rule = true;
  if ((c->stop_kind == STOP_DISCREPANCY || c->stop_kind == STOP_LANDED) && 2.0 * c->J_pred * c->inv_pS <= c->eta) {
    rule = true;
    c->capped = 0;
    // landed stop: shorten this step so that the discrepancy ends in [eta (1 - tol), eta]
    const double Jt = c->eta * (1.0 - 0.5 * c->tol) / (2.0 * c->inv_pS);
    if (c->stop_kind == STOP_LANDED && c->J_pred < Jt && c->J > Jt) {
      c->land_pass = 1;
      c->land_lo = 0.0; c->land_hi = lam;
      c->land_Jlo = c->J; c->land_Jhi = c->J_pred; c->land_Jt = Jt;
      return;                         // the landing passes decide lambda and set done
    }
  }
  const bool stop = rule || kn >= c->max_iter;
  c->capped = stop && !rule;
  if (stop) c->done = 1;
}

// After a landing pass (K8): the candidates lam_i = lo + (i + 1) (hi - lo)/(kLandCand + 1) give
// J(lam_i) = J + Delta J(lam_i).  J is convex along the step and J(lo) > Jt >= J(hi), so the first
// candidate with J <= Jt closes the new bracket.  After the last pass lambda interpolates J
// linearly between the bracket ends; by convexity the chord lies above J, so the stored J_pred
// (= Jt) bounds the true value from above and the discrepancy ends at most eta (1 - tol/2).
__device__ inline void sgp_land_decide(double* trace, CtrlState* c, const double (&dj)[kLandCand]) {
  const double lo = c->land_lo, hi = c->land_hi, h = (hi - lo) / double(kLandCand + 1);
  double nlo = lo, nhi = hi, Jlo = c->land_Jlo, Jhi = c->land_Jhi;
  for (int i = 0; i < kLandCand; ++i) {
    const double Ji = c->J + dj[i];
    if (!(Ji > c->land_Jt)) { nhi = lo + double(i + 1) * h; Jhi = Ji; break; }
    nlo = lo + double(i + 1) * h; Jlo = Ji;
  }
  c->land_lo = nlo; c->land_hi = nhi; c->land_Jlo = Jlo; c->land_Jhi = Jhi;
  c->land_pass += 1;
  if (c->land_pass <= kLandPasses) return;
  const double w = Jlo > Jhi ? (Jlo - c->land_Jt) / (Jlo - Jhi) : 1.0;
  const double lam = nlo + fmin(fmax(w, 0.0), 1.0) * (nhi - nlo);
  const double Jp = Jlo + fmin(fmax(w, 0.0), 1.0) * (Jhi - Jlo);
  c->lambda = lam;
  c->dJ = Jp - c->J;
  c->J_pred = Jp;
  c->R_pred = c->R + reg_delta(c, lam);
  c->land_pass = 0;
  c->done = 1;
  if (c->trace_n >= 1 && c->trace_n <= c->trace_cap) {   // the record sgp_accept wrote
    double* r = trace + size_t(c->trace_n - 1) * kTraceStride;
    r[1] = Jp; r[2] = 2.0 * Jp * c->inv_pS; r[4] = lam;
  }
}
template <bool FP64>
__device__ void ctrl_sgp_land(const ImgDesc& d) {
  __shared__ CtrlState s;
  double* const trace = d.trace;                  // loaded while the partial sums are read
  const CtrlCopy cp(d.ctrl);
  double dj[kLandCand];
  ctrl_sum<kLandCand, FP64>(d, SLOT_ARMX, dj, false);
  cp.to_shared(s);
  if (threadIdx.x == 0) sgp_land_decide(trace, &s, dj);
  CtrlCopy::write_back(s, d.ctrl);
}

template <bool FP64>
__device__ void sgp_lambda_decide(double* trace, CtrlState* c, double gTd, const double (&arm)[kArmMain]) {
  c->gTd = gTd;
  if (!isfinite(gTd)) { c->status = 8; c->done = 2; return; }
  double lam = 1.0;
  const int nl = arm_count(c);
  for (int i = 0; i < nl && i <= c->max_backtracks; ++i) {
    const double dobj = arm[i] + reg_delta(c, lam);   // change of J_0 + R
    const bool ok = FP64 ? (dobj <= c->beta * lam * gTd)
                         : (float(dobj) <= float(c->beta) * float(lam) * float(gTd));
    if (ok) { sgp_accept(trace, c, i, lam, arm[i]); return; }
    lam *= c->theta;
  }
  c->need_more = 1;
}
template <bool FP64>
__device__ __forceinline__ void ctrl_sgp_lambda(const ImgDesc& d, bool dry) {
  __shared__ CtrlState s;
  double* const trace = dry ? nullptr : d.trace;  // both loaded while the partial sums are read
  const bool reg = d.reg_beta > 0.0f;
  const CtrlCopy cp(d.ctrl);
  double g[1], arm[kArmMain], rg[2] = {0.0, 0.0};
  ctrl_sums<1, kArmMain, FP64>(d, SLOT_GTD, false, g, SLOT_ARM, true, arm);
  if (reg) ctrl_sum<2, FP64>(d, SLOT_REG, rg, false);   // f'd, d'd of this direction
  cp.to_shared(s);
  if (threadIdx.x == 0) {
    s.reg_fd = rg[0];
    s.reg_dd = rg[1];
    sgp_lambda_decide<FP64>(trace, &s, g[0], arm);
  }
  if (!dry) CtrlCopy::write_back(s, d.ctrl);
  else __syncthreads();
}
template <bool FP64>
__device__ __noinline__ void ctrl_sgp_lambda_nl(const ImgDesc& d, bool dry) { ctrl_sgp_lambda<FP64>(d, dry); }

template <bool FP64>
__device__ void sgp_lambda_extra_decide(double* trace, CtrlState* c, const double (&arm)[kArmExtra]) {
  const int nl = arm_count(c);
  double lam = 1.0;
  for (int i = 0; i < nl; ++i) lam *= c->theta;
  const double gTd = c->gTd;
  for (int i = 0; i < kArmExtra && nl + i <= 30 && nl + i <= c->max_backtracks; ++i) {
    const double dobj = arm[i] + reg_delta(c, lam);
    const bool ok = FP64 ? (dobj <= c->beta * lam * gTd)
                         : (float(dobj) <= float(c->beta) * float(lam) * float(gTd));
    if (ok) { sgp_accept(trace, c, nl + i, lam, arm[i]); return; }
    lam *= c->theta;
  }
  c->need_more = 0;
  c->status = 6;                      // line search failed: stop at f^(k)
  c->done = 2;
}
template <bool FP64>
__device__ void ctrl_sgp_lambda_extra(const ImgDesc& d) {
  __shared__ CtrlState s;
  double* const trace = d.trace;                  // loaded while the partial sums are read
  const CtrlCopy cp(d.ctrl);
  double arm[kArmExtra];
  ctrl_sum<kArmExtra, FP64>(d, SLOT_ARMX, arm, false);
  cp.to_shared(s);
  if (threadIdx.x == 0) sgp_lambda_extra_decide<FP64>(trace, &s, arm);
  CtrlCopy::write_back(s, d.ctrl);
}

template <bool FP64>
__device__ void rl_decide(double* trace, CtrlState* c, double kl, double rr) {
  const bool updated = c->have_v;
  if (updated) c->k += 1;
  c->have_v = 1;
  // a stop skips the adjoint pass that follows, so v is not available to a resumed run
  if (!isfinite(kl)) { c->status = 8; c->done = 2; c->have_v = 0; return; }
  c->J_prev = c->J;
  c->J = kl;
  if (updated) trace_push(trace, c, c->k, c->J, 0.0, 1.0, 0, 0, 0.0);
  if (c->stop_kind == STOP_MIN_ERROR && c->ftrue_norm2 > 0.0) {
    const double rho = sqrt(rr / c->ftrue_norm2);
    c->rho = rho;
    if (c->k >= 1 && rho > c->rho_prev) { c->done = 2; c->result_prev = 1; c->have_v = 0; return; }
    c->rho_prev = rho;
  }
  bool rule = false;                  // the stop rule itself fired (not only the iteration cap)
  if (updated && c->stop_kind == STOP_CONVERGENCE && fabs(c->J - c->J_prev) <= c->tol * c->J_prev) rule = true;
  if (c->stop_kind == STOP_DISCREPANCY && 2.0 * c->J * c->inv_pS <= c->eta) rule = true;
  const bool stop = rule || c->k >= c->max_iter;
  c->capped = stop && !rule;
  if (stop) { c->done = 2; c->have_v = 0; }
}
// OSEM bookkeeping (Algorithm 2), by one thread: an update h <- w_j h A_j^T r_j was applied when v
// was available; count it (k counts view updates, p per OSEM iteration; f[k & 1] holds h).
__device__ inline void osem_tick(CtrlState* c, int have_v_after) {
  if (threadIdx.x == 0) {
    c->k += c->have_v;
    c->have_v = have_v_after;
  }
}

// real in the last block of the RL ratio pass, dry in the others (as the SGP controllers above)
template <bool FP64>
__device__ __forceinline__ void ctrl_rl(const ImgDesc& d, bool dry) {
  __shared__ CtrlState s;
  double* const trace = dry ? nullptr : d.trace;  // loaded while the partial sums are read
  const CtrlCopy cp(d.ctrl);
  double kl[1], rr[1];
  ctrl_sums<1, 1, FP64>(d, SLOT_KL, true, kl, SLOT_RHO, false, rr);
  cp.to_shared(s);
  if (threadIdx.x == 0) rl_decide<FP64>(trace, &s, kl[0], rr[0]);
  if (!dry) CtrlCopy::write_back(s, d.ctrl);
  else __syncthreads();
}
template <bool FP64>
__device__ __noinline__ void ctrl_rl_nl(const ImgDesc& d, bool dry) { ctrl_rl<FP64>(d, dry); }

}  // namespace sgp
