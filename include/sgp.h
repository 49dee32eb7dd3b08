/*
 * sgp.h -- C ABI of the B300 (sm_103a) Richardson-Lucy / scaled gradient projection (SGP)
 * deconvolution library.
 *
 * The methods are those of Prato, Cavicchioli, Zanni, Boccacci & Bertero, "Efficient
 * deconvolution methods for astronomical imaging: algorithms and IDL-GPU codes":
 *   - the imaging model A_j f = K_j * f with unit-volume PSFs K_j (Sect. 1, Sect. 2.3) and, with a
 *     boundary mask, A_j f = M_S (K_j * (M_R f)), A_j^T y = M_R (K_j (x) (M_S y)) on an extended
 *     domain (Sect. 2.4, Eq. projection / backprojection);
 *   - the KL divergence J_0 (Sect. 1, Eq. KL; Sect. 2.3, Eq. multipleKL) and its gradient
 *     (Eq. KLgrad, multiplegradient, gradientboundary);
 *   - Richardson-Lucy in single, multiple and boundary form (Eq. RL, multipleRL, boundaryRL);
 *   - SGP, Algorithm 1, with the scaled Barzilai-Borwein step lengths (Eq. BB1, BB2), their
 *     safeguards and alternation (Eq. alphadef), the RL scaling (Eq. Dk, Dkbound), the Armijo line
 *     search, the parameter values and adaptive bounds of Sect. 3.2;
 *   - the starting points of Sect. 3.1 and the stopping rules of Sect. 3.3 (fixed number,
 *     Eq. convergence, minimum reconstruction error, Eq. discrepancy).
 *
 * Conventions
 *   - Every pointer documented as "device" is a CUDA device pointer owned by the caller.  The
 *     library copies the inputs it needs (PSFs, data, backgrounds, masks) into the caller's
 *     workspace during the call and keeps no caller pointer afterwards, except the reference object
 *     given to sgp_set_truth, which must stay valid while solves use it.
 *   - Arrays are float32, C-contiguous: a p-view array is p x H x W, an image is H x W.
 *   - Supported sides: H, W in {16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536,
 *     2048} (powers of two and three times powers of two); 1 <= p <= 8 views.
 *   - The workspace (device memory of sgp_workspace_bytes bytes, 256-byte aligned) is owned by
 *     the caller and must outlive the context; the library never allocates device memory.
 *   - `stream` is a cudaStream_t (passed as void*; NULL = legacy default stream).  Calls are
 *     ordered with that stream.  sgp_create, sgp_set_data, kl_value, sgp_get_*, sgp_solve_until
 *     and rl_solve_until synchronise; sgp_set_start, rl_iterate, sgp_iterate, sgp_apply_A and
 *     sgp_apply_AT are asynchronous (a user start f0 is read in stream order).
 *   - Every call returns an sgp_status; sgp_last_error() gives a message for the calling thread.
 *   - A context is not thread safe; use one context per host thread.
 */
#ifndef SGP_B300_H
#define SGP_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SGP_API __attribute__((visibility("default")))
#else
#define SGP_API
#endif

typedef struct sgp_ctx sgp_ctx;

typedef enum {
  SGP_OK = 0,
  SGP_ERR_ARG = 1,              /* invalid argument, missing data, no positive pixel for L1/L2 */
  SGP_ERR_SIZE_UNSUPPORTED = 2, /* H, W or p outside the supported set */
  SGP_ERR_PSF = 3,              /* PSF not finite, sum <= 0, or significantly negative */
  SGP_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  SGP_ERR_WORKSPACE = 5,        /* workspace too small or misaligned */
  SGP_ERR_LINESEARCH = 6,       /* Armijo loop exceeded max_backtracks reductions */
  SGP_ERR_TIMEOUT = 7,          /* iteration cap reached before the stop rule */
  SGP_ERR_NONFINITE = 8,        /* non-finite data, objective or gradient */
  SGP_ERR_STATE = 9             /* call not valid in the current state */
} sgp_status;

enum { SGP_STOP_FIXED = 0, SGP_STOP_CONVERGENCE = 1, SGP_STOP_DISCREPANCY = 2, SGP_STOP_MIN_ERROR = 3,
       SGP_STOP_DISCREPANCY_LANDED = 4 };
/* SGP_STOP_DISCREPANCY_LANDED (SGP only): the discrepancy stop of Sect. 3.3 with the last step
 * shortened so that the final discrepancy lies in [eta (1 - tol), eta] (tol <= 0 means 1e-5):
 * two passes bracket lambda on [0, lambda_accepted] and a chord interpolation picks it; by
 * convexity of J along the step the shortened step still satisfies the Armijo condition.  Runs
 * stopped this way end at the same KL to within tol, whatever their start (the paper stops at
 * the first iterate with D <= eta; this rule is a reading of it, not in the paper). */
enum { SGP_START_ZERO = 0, SGP_START_DATA = 1, SGP_START_CONSTANT = 2, SGP_START_USER = 3 };
enum { SGP_PSF_CENTER = 0, SGP_PSF_CORNER = 1 };

/* One problem: p detected images of an H x W object (Sect. 2.3); has_mask selects boundary-effect
 * correction on the extended domain H x W (Sect. 2.4); psf_origin: SGP_PSF_CENTER = PSF origin at
 * pixel (H/2, W/2), SGP_PSF_CORNER = at (0, 0). */
typedef struct {
  int H, W, p;
  int has_mask;
  int psf_origin;
} sgp_shape;

/* Method parameters; sgp_params_default() gives the values of Sect. 3.2. */
typedef struct {
  double beta;          /* Armijo parameter (1e-4) */
  double theta;         /* backtracking factor (0.4) */
  double alpha0;        /* first step length (1.3) */
  double tau1;          /* alternation threshold tau_1 (0.5) */
  double alpha_min;     /* 1e-5 */
  double alpha_max;     /* 1e5 */
  int M_alpha;          /* BB2 window (3), <= 16 */
  int warmup_iters;     /* iterations using the windowed BB2 before alternating (20) */
  int adaptive_L;       /* 1: L1/L2 from one RL step (Sect. 3.2); 0: use L1, L2 below */
  int max_backtracks;   /* cap on Armijo reductions (30, <= 30) */
  double L1, L2;        /* fixed scaling bounds when adaptive_L == 0 (1e-10, 1e10) */
  double sigma_R;       /* threshold of Eq. (Rdef) for the reconstruction domain R (1e-2) */
  int constraint;       /* 0: f >= 0; 1: f >= 0 and sum f = flux_c (projection in the D^-1 metric) */
  double flux_c;        /* flux for constraint 1; <= 0 means mean over views of sum_S (g - b) */
  int reduce_fp64;      /* 1: FP64 accumulation of KL / BB / Armijo sums (default); 0: plain FP32 */
  int trace_cap;        /* per-problem iteration records kept on the device (4096) */
  double band_tol;      /* PSF band (1e-6): spectrum columns kx whose PSF spectrum entries are all
                         * <= band_tol max|K_hat| (every view) are treated as zero, so the iteration's
                         * row transforms store and load only the band and the column passes process
                         * only it -- for band-limited PSFs (diffraction-limited pupils, whose
                         * optical transfer function vanishes beyond the pupil's autocorrelation)
                         * a large saving; the dropped entries lie below the FP32 transforms' own
                         * rounding.  0 keeps every column. */
  double reg_beta;      /* regularised SGP (Sect. 5 names the extension and its split-gradient scaling;
                         * the regulariser is this library's reading): 0 = the method above (default);
                         * > 0 minimises J_0 + reg_beta/2 ||f||^2 with the split-gradient scaling
                         * D = w c / (1 + reg_beta w c), c = clip(f, L1, L2), the gradient J_0' + reg_beta f;
                         * the Armijo test and the convergence rule use J_0 + R, R = reg_beta/2 ||f||^2,
                         * the discrepancy rules J_0 alone.  RL and OSEM calls return SGP_ERR_ARG. */
} sgp_params;

typedef struct {
  int kind;              /* SGP_STOP_* */
  int max_iter;          /* cap on the number of further iterations */
  double tol;            /* convergence: |J_{k+1} - J_k| <= tol J_k; landed discrepancy: band */
  double eta;            /* discrepancy: stop at the first k with 2 J_0 / (p |S|) <= eta */
} sgp_stop_rule;

typedef struct {
  const float* psfs;     /* device, p x H x W, PSF samples (normalised by the library) */
  const float* b;        /* device, p x H x W backgrounds, or NULL to use b_const */
  float b_const[8];      /* constant background per view */
  const uint8_t* mask;   /* device, H x W, M_S (nonzero on detected pixels); required iff has_mask */
} sgp_inputs;

typedef struct {
  int k;                 /* iterations performed (index of the current iterate) */
  int status;            /* device-side sgp_status of this problem */
  int stopped;           /* 1 when the last stop rule fired */
  int trace_n;           /* number of trace records written */
  double J;              /* J_0 at the current iterate */
  double D;              /* discrepancy 2 J_0 / (p |S|) */
  double L1, L2;         /* scaling bounds in use */
  double alpha, tau, lambda, rho;
  double nS;             /* |S| (pixels of the detected image) */
  double flux_c;         /* constant start value c of Sect. 3.1 */
  int band_cols;         /* spectrum columns processed by the iteration (W/2 = all; see band_tol) */
  double reg;            /* reg_beta/2 ||f||^2 at the current iterate (0 without regularisation) */
} sgp_info;

/* Fill *out with the parameter values of Sect. 3.2. */
SGP_API void sgp_params_default(sgp_params* out);

/* Workspace bytes needed for n problems of the given shapes (params may be NULL = defaults). */
SGP_API size_t sgp_workspace_bytes(int n, const sgp_shape* shapes, const sgp_params* params);

/* Create a context for n problems that advance together (n = 1 for a single problem).
 * For each problem: validate the shape, normalise each PSF to unit volume over the (extended)
 * domain (Sect. 2.4), move its origin to (0, 0), store its spectrum, copy the backgrounds, and for
 * boundary problems compute alpha_j = K_j (x) M_S, R = {alpha_j >= sigma_R}, M_R / alpha
 * (Eq. Rdef; reading: alpha_j without the garbled factor g).
 * Errors: SGP_ERR_ARG, SGP_ERR_SIZE_UNSUPPORTED, SGP_ERR_PSF, SGP_ERR_WORKSPACE, SGP_ERR_CUDA. */
SGP_API sgp_status sgp_create_batch(sgp_ctx** out, int n, const sgp_shape* shapes, const sgp_inputs* inputs,
                            const sgp_params* params, void* workspace, size_t workspace_bytes, void* stream);

/* Single-problem form of sgp_create_batch. b: device p x H x W or NULL; b_const: host array of p
 * constant backgrounds (used when b is NULL); mask: device H x W or NULL. */
SGP_API sgp_status sgp_create(sgp_ctx** out, const sgp_shape* shape, const float* psfs, const float* b,
                      const float* b_const, const uint8_t* mask, const sgp_params* params,
                      void* workspace, size_t workspace_bytes, void* stream);

/* Detected images g (device, p x H x W, counts >= 0) of problem `image`; pixels outside S are
 * ignored.  Sets the constant starting point of Sect. 3.1 unless sgp_set_start is called later.
 * Errors: SGP_ERR_NONFINITE for negative or non-finite data, SGP_ERR_ARG. */
SGP_API sgp_status sgp_set_data(sgp_ctx* ctx, int image, const float* g);

/* Starting point (Sect. 3.1): SGP_START_ZERO, SGP_START_DATA (g_1), SGP_START_CONSTANT
 * (mean over views of sum_S (g - b) / |S|, on R), SGP_START_USER (device H x W f0, clipped at 0
 * and restricted to R).  Resets the iteration count. */
SGP_API sgp_status sgp_set_start(sgp_ctx* ctx, int image, int mode, const float* f0);

/* Reference object for the minimum-reconstruction-error stop (Sect. 3.3); device H x W, must stay
 * valid while solves run; NULL clears it. */
SGP_API sgp_status sgp_set_truth(sgp_ctx* ctx, int image, const float* f_true);

/* n Richardson-Lucy iterations of every problem (Eq. RL, multipleRL, boundaryRL).  Asynchronous. */
SGP_API sgp_status rl_iterate(sgp_ctx* ctx, int n);

/* n SGP iterations (Algorithm 1) of every problem.  Asynchronous. */
SGP_API sgp_status sgp_iterate(sgp_ctx* ctx, int n);

/* n OSEM iterations (ordered-subset expectation maximisation, Sect. 2.3, Algorithm 2) of every
 * problem, from its current iterate: each iteration cycles over the views j = 1..p in order with
 * h <- h o A_j^T (g_j / (A_j h + b_j)) (Eq. OSEMstep), or, with a boundary mask,
 * h <- (M_R / alpha_j) o h o A_j^T (...) (Eq. boundaryOSEM), alpha_j = K_j (x) M_S.  Four passes per
 * view (4p transforms per iteration).  With p = 1 it is RL.  Afterwards kl_value gives J_0 of the
 * result and sgp_get_f the result; sgp_get_info's k counts view updates (p per iteration).  No
 * stop rule (the paper runs OSEM for a given number of iterations).  Needs problems of one size
 * (SGP_ERR_STATE for a context of mixed sizes).  Asynchronous, except that the first call after
 * set-up may tune the row tile (see sgp_get_tile). */
SGP_API sgp_status osem_iterate(sgp_ctx* ctx, int n);

/* Iterate SGP (resp. RL) on every problem until its stop rule fires or max_iter further
 * iterations; iters (n ints, may be NULL) receives each problem's iteration count.
 * Returns SGP_ERR_TIMEOUT if some problem reached max_iter before a non-FIXED rule fired, or the
 * first device-side error status. */
SGP_API sgp_status sgp_solve_until(sgp_ctx* ctx, const sgp_stop_rule* rule, int* iters);
SGP_API sgp_status rl_solve_until(sgp_ctx* ctx, const sgp_stop_rule* rule, int* iters);

/* J_0 (FP64) at the current iterate of problem `image` (Eq. KL / multipleKL). */
SGP_API sgp_status kl_value(sgp_ctx* ctx, int image, double* out);

/* Copy the current iterate (the returned one after a minimum-error stop) to dst (device H x W). */
SGP_API sgp_status sgp_get_f(sgp_ctx* ctx, int image, float* dst);

/* Per-iteration records, 8 doubles each: k, J_0, discrepancy, alpha, lambda, backtracks,
 * branch (0 alpha_0, 1 BB1, 2 windowed BB2), grad'd.  out: host, cap records. */
SGP_API sgp_status sgp_get_trace(sgp_ctx* ctx, int image, double* out, int cap, int* count);

SGP_API sgp_status sgp_get_info(sgp_ctx* ctx, int image, sgp_info* out);

/* Operators of problem `image` (Eq. projection / backprojection): out_j = A_j f for every view
 * (out: device p x H x W); out = sum_j A_j^T y_j (y: device p x H x W, out: device H x W).
 * They use the problem's iteration buffers as scratch: the next iterate call re-initialises the
 * iteration from the current iterate.  Asynchronous. */
SGP_API sgp_status sgp_apply_A(sgp_ctx* ctx, int image, const float* f, float* out);
SGP_API sgp_status sgp_apply_AT(sgp_ctx* ctx, int image, const float* y, float* out);

/* Measurement aid: run `iters` SGP iterations launching each pass separately, bracketed by CUDA
 * events on the library's stream, and return the mean duration in ms of the 7 passes of an
 * iteration in ms_out[0..6]: K1 update + ratio (+ iteration controller), column A^T, K3 gradient +
 * BB sums (+ step-length controller), K4 projection, column A, K6 A d + Armijo (+ line-search
 * controller), extra Armijo (+ its controller; returns at once unless needed).  n_out >= 7;
 * SGP_ERR_ARG for a flux-constrained context.  The iterations advance the state; the next solve
 * restarts from the current iterate. */
SGP_API sgp_status sgp_time_passes(sgp_ctx* ctx, int iters, double* ms_out, int n_out);

/* Number of kernels this context has enqueued so far (graph launches count their nodes). */
SGP_API long long sgp_launch_count(sgp_ctx* ctx);

/* Row tile of the hot row passes (contexts whose problems share one size).  A row pass runs one
 * block per work item of R image rows, T = 256 / R_max threads per row, where R_max is the tile of
 * a 256-thread block.  At the first iterate/solve call an autotuner times the projection pass for
 * R = R_max, R_max/2, ... down to 32-thread blocks and keeps the fastest (the choice is shared by
 * every context of the same H, W, p in the process).  sgp_get_tile reports R and the block size
 * (R = 0 and 256 for mixed-size contexts); sgp_set_tile forces R (SGP_ERR_ARG if R is not a
 * candidate, SGP_ERR_STATE for a mixed-size context), drops the captured graphs and makes the next
 * iterate/solve call re-initialise from the current iterate.  Partial sums are grouped per work
 * item, so results depend on R at rounding level. */
SGP_API sgp_status sgp_get_tile(sgp_ctx* ctx, int* rows_per_item, int* threads_per_block);
SGP_API sgp_status sgp_set_tile(sgp_ctx* ctx, int rows_per_item);

/* Convolution without any device allocation, for callers that cannot allocate device memory --
 * for example code running where cudaMalloc is unavailable or forbidden (inside a captured region
 * of another framework, under a strict memory budget owned by someone else, or in a process that
 * must not grow its device footprint after start-up).  It computes the same result as sgp_apply_A
 * (transpose = 0: out = K * f) or sgp_apply_AT (transpose = 1: out = K (x) f) of a periodic
 * single-view problem with PSF `psf` (normalised here to unit sum; psf_origin as in sgp_shape),
 * without a context or workspace.  The paper has no counterpart of this entry point.
 *   - psf, f, out: device H x W float32 arrays owned by the caller.
 *   - Limit: H * W <= 262144 (e.g. 512 x 512); larger sizes return SGP_ERR_SIZE_UNSUPPORTED.
 *   - Scratch: a fixed 3.2 MB array inside the library, held on every GPU that loads the library
 *     until the process exits.  Every region of it is written before it is read, so no clearing
 *     is needed between calls.  All calls share it: calls whose GPU work overlaps (other streams,
 *     other host threads) race and must be serialised by the caller.
 *   - The first call on a device looks up the address of that array (and initialises the library
 *     on the device); concurrent first calls from several host threads are serialised.
 *   - Every call synchronises `stream` once (to read the PSF sum) and copies small tables from
 *     host memory, so it must never be called while `stream` is being captured into a CUDA
 *     graph: it then returns SGP_ERR_STATE without doing anything.
 *   - Allocates nothing.  SGP_ERR_ARG for a device ordinal of 64 or more. */
SGP_API sgp_status sgp_convolve_noalloc(const float* psf, const float* f, float* out, int H, int W,
                                        int psf_origin, int transpose, void* stream);

/* Mosaic of boundary-corrected reconstructions (Sect. 4, second experiment; Table 2, Table 6).
 * An H x W image is covered by ny x nx partially overlapping sub-domains of sub_h x sub_w pixels;
 * each sub-image is merged by zero padding into an ext_h x ext_w array (sub-image centred at offset
 * floor((ext - sub)/2), M_S = 1 on it), reconstructed there with the boundary-effect correction
 * (a context of ny * nx boundary problems advancing together), and the mosaic keeps one
 * non-overlapping piece of each reconstruction.  Along an axis of N pixels with n sub-domains of
 * s pixels: sub-domain k = [floor(k (N - s)/(n - 1)), + s) and piece k = [floor(k N/n),
 * floor((k + 1) N/n)) (the paper's example: 256 -> 2 x 160 -> pieces of 128).  1 <= ny, nx <= 16;
 * sub <= the image and <= ext; every piece must lie inside its sub-domain (else SGP_ERR_ARG). */
typedef struct {
  int H, W;             /* image */
  int ny, nx;           /* sub-domains per axis */
  int sub_h, sub_w;     /* sub-domain size */
  int ext_h, ext_w;     /* padded array (a supported side for the reconstruction context) */
} sgp_mosaic;

/* Checks the geometry and writes 4 (ny + nx) ints to out (may be NULL): for ky = 0..ny-1 the
 * sub-domain start, end, piece start, end along H, then the same for kx along W. */
SGP_API sgp_status sgp_mosaic_geometry(const sgp_mosaic* m, int* out);

/* g: device p x H x W -> tiles: device (ny nx) x p x ext_h x ext_w (zero-padded sub-images, tile
 * t = ky nx + kx) and masks: device (ny nx) x ext_h x ext_w uint8 M_S.  Asynchronous on stream. */
SGP_API sgp_status sgp_mosaic_split(const sgp_mosaic* m, int p, const float* g, float* tiles, uint8_t* masks,
                                    void* stream);

/* recs: device (ny nx) x ext_h x ext_w reconstructions -> f: device H x W mosaic.  Asynchronous. */
SGP_API sgp_status sgp_mosaic_stitch(const sgp_mosaic* m, const float* recs, float* f, void* stream);

/* Verification aid for the precision of the library's sums (the KL value J_0 of Eq. KL, the
 * numerators and denominators of the scaled BB rules Eq. BB1 / BB2, the Armijo differences of
 * Algorithm 1, step 5).  For i < n it computes the pixel term t_i of one kind with the same device
 * functions the iteration passes use, writes it to terms[i] (device float32, may be NULL) and sums
 * the t_i with the passes' reduction: per-thread accumulation over 32 terms, warp and block sums,
 * a fixed-order sum of the block partials.  reduce_fp64 = 1 selects the mixed variant (error-free
 * FP32 two-sum accumulation and FP32 pairs, as with sgp_params.reduce_fp64 = 1), 0 plain FP32.
 *   kind SGP_SUM_VALUES: t = a (any float32 values)
 *        SGP_SUM_KL:     t = g ln(g/u) + u - g with g = a, u = b (u = A f + background)
 *        SGP_SUM_ARMIJO: t = lambda A d - g ln(1 + lambda A d / u) with g = a, u = b, A d = c
 *        SGP_SUM_BB0..3: s^2 / D^2, s z / D, s z D, z^2 D^2 with s = a, z = b, D = c (0 where D <= 0)
 * a, b, c: device float32 arrays of n values (b, c unused by the kinds that do not name them).
 * out: host, receives the sum as FP64.  workspace: device, 256-byte aligned, at least
 * sgp_sum_terms_workspace_bytes(n) bytes, owned by the caller.  Synchronises `stream`.
 * Errors: SGP_ERR_ARG, SGP_ERR_WORKSPACE, SGP_ERR_SIZE_UNSUPPORTED, SGP_ERR_CUDA. */
enum { SGP_SUM_VALUES = 0, SGP_SUM_KL = 1, SGP_SUM_ARMIJO = 2, SGP_SUM_BB0 = 3, SGP_SUM_BB3 = 6 };
SGP_API size_t sgp_sum_terms_workspace_bytes(size_t n);
SGP_API sgp_status sgp_sum_terms(int kind, int reduce_fp64, const float* a, const float* b, const float* c,
                                 size_t n, double lambda, float* terms, double* out, void* workspace,
                                 size_t ws_bytes, void* stream);

/* Release the context (not the workspace). */
SGP_API sgp_status sgp_destroy(sgp_ctx* ctx);

/* Message of the last error on the calling thread ("" if none). */
SGP_API const char* sgp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGP_B300_H */
