// Device-resident problem state shared by the kernels and the host runtime.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace sgp {

constexpr int kMaxViews = 8;        // p <= 8 views per problem
constexpr int kMaxHist = 16;        // >= M_alpha
constexpr int kPartStride = 56;     // doubles of partial sums per row item
constexpr int kTraceStride = 8;     // doubles per trace record
constexpr int kRowBlock = 256;      // threads of every row-pass block
constexpr int kColBlock = 512;      // threads of every column-pass block
constexpr int kCtrlBlock = 256;     // threads of the controller blocks

// Programmatic dependent launch: the hot passes are launched so that a pass's launch is processed
// while the previous pass drains; every such kernel waits (in hardware, griddepcontrol.wait) until
// the previous grid has completed and its memory is visible before it reads anything.  (Letting
// the successor's blocks become resident early measured slower at the start of a pass, 5.54 ms
// against 4.66 ms for the 2048^2 solve, and no faster before the controller tail, 4.68 ms.)
// Without the launch attribute the wait returns at once.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// partial-sum slots (per row item)
enum Slot {
  SLOT_KL = 0,        // sum of KL terms (J_0)
  SLOT_RHO = 1,       // sum (f - f_true)^2
  SLOT_BB = 2,        // 4 slots: s'D^-2 s, s'D^-1 z, s'D z, z'D^2 z
  SLOT_GTD = 6,       // grad' d
  SLOT_FLUX = 7,      // sum f
  SLOT_ARM = 8,       // kArmMain slots: Delta J(theta^i), i < arm_nl (main pass)
  SLOT_ARMX = 12,     // kArmExtra slots: Delta J(theta^i), i = arm_nl..30 (only when needed)
  SLOT_MIN = 42,      // min over positive pixels (set-up)
  SLOT_MAX = 43,      // max (set-up)
  SLOT_PROJ = 44,     // flux projection search sums (5)
  SLOT_REG = 50,      // regularised SGP: 2 slots, f'd and d'd (Armijo change of the Tikhonov term)
  SLOT_FSQ = 52,      // regularised SGP set-up: f'f of the starting point
};
// The main Armijo pass evaluates arm_count() step lengths 1, theta, ..: one after an iteration that
// accepted lambda = 1, two after one backtrack, kArmMain after more.
constexpr int kArmMain = 4;
constexpr int kArmExtra = 30;           // theta^1 .. theta^30 at most in the extra pass
constexpr int kFluxCand = 16;       // candidate mu values per flux-search pass (slots SLOT_ARMX..)
constexpr int kFluxPasses = 5;

enum ColMode { COL_KHAT = 0, COL_1TOP = 1, COL_1TOP_CONJ = 2, COL_PTO1 = 3, COL_PTOV = 4 };

enum StopKind { STOP_FIXED = 0, STOP_CONVERGENCE = 1, STOP_DISCREPANCY = 2, STOP_MIN_ERROR = 3, STOP_LANDED = 4 };
constexpr int kLandCand = kArmExtra;   // step lengths per landing pass (slots SLOT_ARMX..)
constexpr int kLandPasses = 2;

// Controller state of one problem (in the workspace; read by every hot kernel).
struct CtrlState {
  int k;            // index of the current iterate f^(k)
  int fresh;        // SGP: 1 when f[k&1] is current, 0 when f^(k+1) = f^(k) + lambda d is pending
  int done;         // 0 running; 1 stop decided, final SGP update pending; 2 stopped
  int status;       // device-side status (sgp_status code), 0 = OK
  int need_more;    // Armijo: no lambda of the main pass accepted
  int have_v;       // RL: spectrum plane 0 holds sum_j A_j^T r_j of the current iterate
  int branch;       // 0: alpha_0, 1: BB1, 2: windowed BB2
  int backtracks;
  int result_prev;  // min-error stop: the result is the previous iterate f[(k-1)&1]
  int hist_n;
  int trace_n, trace_cap;
  int stop_kind, max_iter;
  int M_alpha, warmup, max_backtracks, fp64;
  int constraint;   // 0 non-negativity, 1 + flux
  int proj_pass;    // flux projection search pass
  unsigned arrive;  // blocks of the current row pass that have stored their partial sums
  int arm_nl;       // step lengths of the main Armijo pass (1, 2 or kArmMain; 0 before the first)
  int land_pass;    // landed discrepancy stop: 0 idle; n > 0 landing the last step, n - 1 passes done
  int f_pending;    // SGP: K1 left f^(k+1) = f^(k) + lambda d to the gradient pass, which forms it
                    // from f^(k) and grad^(k) and stores it (see f_update_in_k1)
  int capped;       // 1 when the last stop came from the iteration cap, not from the stop rule
  double land_lo, land_hi, land_Jlo, land_Jhi, land_Jt;   // bracket of lambda, J at its ends, target
  double J;         // J_0 at the current iterate
  double J_pred;    // J_0 at the accepted trial point
  double J_prev;    // RL: J_0 at the previous iterate
  double alpha, alpha_prev, tau, lambda, gTd, dJ, mu, rho_prev, rho;
  double L1, L2;
  double hist[kMaxHist];
  double beta, theta, alpha0, tau1, alpha_min, alpha_max;
  double tol, eta, inv_pS, ftrue_norm2, flux_c;
  double mu_lo, mu_hi, phi_lo, phi_hi;
  double reg_beta;  // weight of the Tikhonov term beta/2 ||f||^2 (0: the unregularised method)
  double R, R_pred; // beta/2 ||f||^2 at the current iterate and at the accepted trial point
  double reg_fd, reg_dd;   // f'd and d'd of the current direction
  double scratch[8];
};
// The pending SGP update f^(k+1) = f^(k) + lambda d (Alg. 1, step 6) is applied by K1 when the stop
// is already decided (the final update) or the minimum-error rule needs f^(k+1) in K1; otherwise
// by the gradient pass K3, which reads f^(k) and grad^(k) anyway, so K1 reads neither.  `done` is
// the value at K1's start.
__host__ __device__ inline bool f_update_in_k1(const CtrlState* c, int done) {
  return done == 1 || c->stop_kind == STOP_MIN_ERROR;
}
__host__ __device__ inline int arm_count(const CtrlState* c) {
  return c->arm_nl == 1 || c->arm_nl == 2 || c->arm_nl == kArmMain ? c->arm_nl : 2;
}

// One problem (p views of an H x W object) as the kernels see it.  Arrays are FP32 row-major with
// P = H*W elements per plane; spectra are H x W/2 complex (the real DC and Nyquist columns of the
// row transform share column 0 as real and imaginary part), i.e. also P floats per plane.
struct ImgDesc {
  int H, W, p, boundary;
  int row_item0, n_row_items;   // this problem's items in the row-item list (image, row0)
  int rv_item0, n_rv_items;     // ... and in the row-view list (image, row0 | view << 16)
  int rpi;                      // image rows per row item
  int cb;                       // spectrum columns in the PSF band (<= W/2): the hot row passes store
                                // and load only columns < cb, the others are zero (band-limited PSF)
  int dry_row, dry_rv;          // 1: the passes over the row (row-view) list run their controller dry
                                // in the blocks that arrive before the last one (control.cuh)
  float w_scalar;               // periodic: 1/p (RL factor, SGP scaling factor)
  float a1_scalar;              // periodic: p (= sum_j A_j^T 1)
  float reg_beta;               // regularised SGP: weight of beta/2 ||f||^2 (0: none)
  float bs[kMaxViews];          // constant backgrounds (used when b == nullptr)
  size_t P;
  float* f[2];                  // iterate ping-pong
  float* grad[2];               // gradient ping-pong
  float* u;                     // p planes: A_j f (without b)
  float* Ad;                    // p planes: A_j d
  float* g;                     // p planes: data; -1 marks pixels outside S (boundary mode)
  const float* b;               // p planes or nullptr
  const float* w;               // boundary: M_R / alpha (0 outside R); nullptr when periodic
  const float* wv;              // boundary: p planes M_R / alpha_j (OSEM weights); nullptr when periodic
  float* spec;                  // (p+1) planes of packed spectra: plane 0, then views 1..p
  const float* ftrue;           // min-error stop only
  CtrlState* ctrl;
  double* part;                 // n_row_items x kPartStride (row-list passes)
  double* partv;                // n_rv_items x kPartStride (row-view-list passes)
  double* trace;                // trace_cap x kTraceStride
};

// A column-pass job: one problem's spectrum planes and PSF spectra.
struct ColJob {
  const float2* in;     // nin planes (plane_stride apart)
  float2* out;          // nout planes
  const float2* khat;   // p planes H x M (column 0 holds P = (K0 + KM)/2)
  float2* khatq;        // p columns of H: Q = (K0 - KM)/2 (written by the spectrum set-up pass)
  int H, M, nin, nout;
  size_t plane_stride;  // float2 elements between planes (= H*M)
  const CtrlState* ctrl;  // skip when ctrl->done >= 1 (nullptr: always run)
  float scale;          // spectrum set-up: 1/(H*M*sum K)
  int corner;           // spectrum set-up: PSF origin already at (0,0)
};

}  // namespace sgp
