// Host runtime and C ABI: workspace layout, set-up passes, iteration sequencing (captured into
// CUDA graphs), stop-rule polling and result access.  Declarations and contracts: include/sgp.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sgp.h"
#include "ctrl.cuh"
#include "mosaic.cuh"
#include "registry.h"
#include "state.cuh"
#include "sumcheck.cuh"

using namespace sgp;

namespace {

thread_local std::string g_err;

sgp_status fail(sgp_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CU(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(SGP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

// ------------------------------------------------------------------------------ registry
Registry g_reg;
bool g_reg_ready = false;

void register_all(Registry& R) {
  memset(&R, 0, sizeof(R));
  register_small(R);
  register_mid(R);
  register_mid_b(R);
  register_large(R);
  register_large_b(R);
  register_multi_sgp_a(R);
  register_multi_sgp_b(R);
  register_multi_armx_f(R);
  register_multi_armx_d(R);
  register_multi_land_f(R);
  register_multi_land_d(R);
  register_multi_rest(R);
}
bool g_dev_ready[64] = {false};

sgp_status ensure_device_ready(int dev) {
  if (!g_reg_ready) {
    register_all(g_reg);
    g_reg_ready = true;
  }
  if (dev < 0 || dev >= 64) return fail(SGP_ERR_CUDA, "device index out of range");
  if (g_dev_ready[dev]) return SGP_OK;
  // twiddle tables exp(-2 pi i q / L) for every supported length, computed in double
  static const int lens[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048};
  std::vector<float2> tab(kTwiddleTotal);
  for (int L : lens) {
    const int off = tw_offset(L);
    for (int q = 0; q < L; ++q) {
      const double a = -2.0 * M_PI * double(q) / double(L);
      tab[off + q] = make_float2(float(cos(a)), float(sin(a)));
    }
  }
  for (int q = 0; q < 32; ++q)   // the four-step table, lane-fastest
    for (int lane = 0; lane < 32; ++lane) {
      const double a = -2.0 * M_PI * double(lane * q) / 1024.0;
      tab[kTw4Offset + 32 * q + lane] = make_float2(float(cos(a)), float(sin(a)));
    }
  for (int i = 0; i < kTwiddleUnits; ++i)
    if (g_reg.twiddle_init[i]) CU(g_reg.twiddle_init[i](tab.data()));
  for (int op = 0; op < ROP_COUNT; ++op)
    for (int f = 0; f < 2; ++f)
      if (g_reg.row_multi[op][f])
        CU(cudaFuncSetAttribute(g_reg.row_multi[op][f], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(g_reg.row_multi_smem)));
  for (int m = 0; m < 3; ++m)
    CU(cudaFuncSetAttribute(g_reg.col_multi[m], cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(g_reg.col_multi_smem)));
  for (int s = 0; s < kNumSides; ++s) {
    for (int op = 0; op < ROP_COUNT; ++op)
      for (int f = 0; f < 2; ++f)
        CU(cudaFuncSetAttribute(g_reg.row[op][f][s], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(g_reg.row_smem[s])));
    for (int m = 0; m < kColModes; ++m)
      CU(cudaFuncSetAttribute(g_reg.col[m][s], cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(g_reg.col_smem[s])));
  }
  for (int m = 0; m < kColModes; ++m)
    CU(cudaFuncSetAttribute(g_reg.col_narrow[m], cudaFuncAttributeMaxDynamicSharedMemorySize,
                            int(g_reg.col_narrow_smem)));
  g_dev_ready[dev] = true;
  return SGP_OK;
}

// ------------------------------------------------------------------------------ workspace carving
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int rows_per_item(int W) { return g_reg.row_rows[side_index(W)]; }
// Rows per work item of the hot row passes: the autotuner tries R_max / 2^k (R_max the rows of a
// 256-thread block) down to blocks of 32 threads (T = 256 / R_max threads per row).
int rows_min(int W) { return std::max(1, rows_per_item(W) / 8); }
int cols_per_item(int H) { return g_reg.col_cols[side_index(H)]; }

struct Layout {
  std::vector<ImgDesc> d;              // per problem
  std::vector<float*> khat, khatq;     // per problem (p planes each)
  std::vector<float*> bcopy;           // per problem (nullptr when constant backgrounds)
  std::vector<double*> scratch;        // per problem 64 doubles
  std::vector<uint8_t*> mS;            // per problem M_S bytes (boundary problems)
  CtrlState* ctrl = nullptr;
  ImgDesc* d_imgs = nullptr;
  int2* d_row = nullptr;               // row list
  int2* d_rv = nullptr;                // row-view list
  int2* d_rvo = nullptr;               // row-view list, view-major over the problems (OSEM sub-steps)
  int2* d_colv = nullptr;              // column list with views (1 -> p passes)
  int2* d_colvo = nullptr;             // the same, view-major over the problems (OSEM sub-steps)
  int2* d_colvb = nullptr;             // column list with views, PSF band only (hot passes)
  int2* d_colb = nullptr;              // column list (p -> 1), PSF band only (hot passes)
  int n_colvb = 0, n_colb = 0;
  int2* d_col = nullptr;               // column list (p -> 1 passes)
  int2* d_colk = nullptr;              // column list of the PSF spectrum jobs
  ColJob* d_jobs = nullptr;            // 5 jobs per problem: A, AT, CONJ, A_raw, AT_raw, then p KHAT jobs
  int* d_flag = nullptr;
  size_t bytes = 0;
  int n_row = 0, n_rv = 0, n_colv = 0, n_col = 0, n_colk = 0, n_jobs = 0;
  int cap_row = 0, cap_rv = 0;         // capacity of the row lists (smallest tile)
  int cap_colb = 0, cap_colvb = 0;     // capacity of the band column lists (smallest column tile)
};

// Count items and carve every array (base == nullptr: only measure).
void plan_layout(char* base, int n, const sgp_shape* sh, int trace_cap, const bool* has_b, Layout& L) {
  Carver cv{base};
  L.d.assign(n, ImgDesc{});
  L.khat.assign(n, nullptr);
  L.khatq.assign(n, nullptr);
  L.bcopy.assign(n, nullptr);
  L.scratch.assign(n, nullptr);
  L.mS.assign(n, nullptr);
  L.n_row = L.n_rv = L.n_colv = L.n_col = L.n_colk = 0;
  L.cap_row = L.cap_rv = 0;
  L.cap_colb = L.cap_colvb = 0;
  for (int i = 0; i < n; ++i) {
    const int H = sh[i].H, W = sh[i].W, p = sh[i].p;
    const size_t P = size_t(H) * W;
    ImgDesc& d = L.d[i];
    d.H = H; d.W = W; d.p = p; d.boundary = sh[i].has_mask ? 1 : 0; d.P = P;
    const int rpi = rows_per_item(W), cpi = cols_per_item(H), M = W / 2;
    d.rpi = rpi;
    d.cb = M;
    const int nr = (H + rpi - 1) / rpi, nc = (M + cpi - 1) / cpi;
    const int ncap = (H + rows_min(W) - 1) / rows_min(W);   // item capacity for the smallest tile
    d.row_item0 = 0; d.n_row_items = nr;      // indices within the problem's own range
    d.rv_item0 = 0; d.n_rv_items = nr * p;
    L.n_row += nr; L.n_rv += nr * p; L.n_col += nc; L.n_colv += nc * p; L.n_colk += nc * p;
    L.cap_row += ncap; L.cap_rv += ncap * p;
    // the band lists may use the narrow column tile (set_band): room for its item count
    const int cpi_b = H == kNarrowSide ? std::min(cpi, g_reg.col_narrow_cols) : cpi;
    const int ncb = (M + cpi_b - 1) / cpi_b;
    L.cap_colb += ncb; L.cap_colvb += ncb * p;
    d.f[0] = cv.take<float>(P); d.f[1] = cv.take<float>(P);
    d.grad[0] = cv.take<float>(P); d.grad[1] = cv.take<float>(P);
    d.u = cv.take<float>(P * p);
    d.Ad = cv.take<float>(P * p);
    d.g = cv.take<float>(P * p);
    L.bcopy[i] = (has_b && has_b[i]) ? cv.take<float>(P * p) : nullptr;
    d.b = L.bcopy[i];
    d.w = d.boundary ? cv.take<float>(P) : nullptr;
    d.wv = d.boundary ? cv.take<float>(P * p) : nullptr;
    d.spec = cv.take<float>(P * (p + 1));
    L.khat[i] = cv.take<float>(P * p);
    L.khatq[i] = cv.take<float>(size_t(2) * H * p);
    d.part = cv.take<double>(size_t(ncap) * kPartStride);
    d.partv = cv.take<double>(size_t(ncap) * p * kPartStride);
    d.trace = cv.take<double>(size_t(trace_cap) * kTraceStride);
    L.scratch[i] = cv.take<double>(64);
    L.mS[i] = d.boundary ? cv.take<uint8_t>(P) : nullptr;
  }
  L.ctrl = cv.take<CtrlState>(n);
  for (int i = 0; i < n; ++i) L.d[i].ctrl = L.ctrl ? L.ctrl + i : nullptr;
  L.d_imgs = cv.take<ImgDesc>(n);
  L.d_row = cv.take<int2>(L.cap_row);
  L.d_rv = cv.take<int2>(L.cap_rv);
  L.d_rvo = cv.take<int2>(L.cap_rv);
  L.d_colv = cv.take<int2>(L.n_colv);
  L.d_colvo = cv.take<int2>(L.cap_colvb);
  L.d_colvb = cv.take<int2>(L.cap_colvb);
  L.d_colb = cv.take<int2>(L.cap_colb);
  L.d_col = cv.take<int2>(L.n_col);
  L.d_colk = cv.take<int2>(L.n_colk);
  int nj = 0;
  for (int i = 0; i < n; ++i) nj += 5 + sh[i].p;
  L.n_jobs = nj;
  L.d_jobs = cv.take<ColJob>(nj);
  L.d_flag = cv.take<int>(16);
  L.bytes = cv.off + 256;
}

}  // namespace

// ------------------------------------------------------------------------------ context
struct sgp_ctx {
  int device = 0;
  int n = 0;
  cudaStream_t s = nullptr;        // internal stream (graphs are captured on it)
  cudaStream_t user = nullptr;     // caller's stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_hctrl = nullptr;  // recorded after each upload from h_ctrl (reset_ctrl)
  sgp_params prm;
  std::vector<sgp_shape> sh;
  Layout L;
  int H = 0, W = 0, p = 0;         // geometry of problem 0 (every problem has the same p)
  bool mixed = false;              // problems of different sides: multi-size kernels
  int fp64 = 1;
  // host mirrors
  std::vector<int2> row, rv, colv, col, colk;
  std::vector<int2> rvo, colvo;    // view-major lists of the OSEM sub-steps (uniform contexts)
  std::vector<int> order;          // problems, largest first (the order of their items)
  int rpi_hot = 0;                 // rows per item of the hot row passes (uniform sizes)
  int row_threads = kRowBlock;     // threads per block of the hot row passes
  size_t row_smem_hot = 0;
  bool tuned = false;
  std::vector<ColJob> jobs;        // per problem: [A, AT, CONJ, A_raw, AT_raw, KHAT x p]
  std::vector<int> job_base;
  std::vector<int> colv_begin, colv_count, col_begin, col_count;
  std::vector<double> c_const;     // constant start per problem
  std::vector<double> nS;          // |S| per problem
  std::vector<int> has_data;
  std::vector<const float*> truth;
  std::vector<double> ftrue_n2;    // ||f_true||^2 per problem (0 without one), as set_truth computed it
  std::vector<int> start_in_f0;    // 1: a new start was written to f[0] since the last set-up
  int mode = 0;                    // 0 not prepared, 1 SGP, 2 RL, 3 OSEM
  cudaGraphExec_t g_sgp = nullptr, g_rl = nullptr;   // graph_units iterations (fixed counts)
  cudaGraphExec_t g_osem = nullptr;  // one OSEM iteration (p sub-steps)
  // solve loops: a WHILE node around one iteration and the loop condition (run_until)
  cudaGraphExec_t gl_sgp = nullptr, gl_rl = nullptr, gl_land = nullptr;
  cudaGraphConditionalHandle hl_sgp = 0, hl_rl = 0, hl_land = 0;
  int graph_units = 8;
  int loop_cap = 0;                // iteration cap captured in the solve loop graphs
  bool col_narrow = false;         // the iteration's column passes use the narrow variant (set_band)
  long long launches = 0;          // kernels enqueued (graph nodes counted per graph launch)
  CtrlState* h_ctrl = nullptr;     // pinned mirror of the controller array
};

namespace {

// ---- launch helpers -----------------------------------------------------------------------------
// launch counter of the context this host thread is driving: set by enter(), cleared by leave()
// and by sgp_destroy() of that context, so it never outlives the context; the entry points that
// drive no context launch with it cleared
thread_local long long* g_launch_counter = nullptr;

sgp_status launch(const void* fn, int grid, int block, size_t smem, cudaStream_t s, void** args) {
  if (grid <= 0) return SGP_OK;
  CU(cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, s));
  if (g_launch_counter) ++*g_launch_counter;
  return SGP_OK;
}
// Launch of a hot pass (its kernel starts with pdl_enter): programmatic dependent launch, so its
// blocks may be scheduled while the previous pass drains.
sgp_status launch_pdl(const void* fn, int grid, int block, size_t smem, cudaStream_t s, void** args) {
  if (grid <= 0) return SGP_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CU(cudaLaunchKernelExC(&cfg, fn, args));
  if (g_launch_counter) ++*g_launch_counter;
  return SGP_OK;
}

sgp_status row_pass(sgp_ctx* c, RowOp op, bool view_list, int extra = -1) {
  const int si = side_index(c->W);
  const void* fn = c->mixed ? g_reg.row_multi[op][c->fp64] : g_reg.row[op][c->fp64][si];
  const size_t smem = c->mixed ? g_reg.row_multi_smem : c->row_smem_hot;
  const int threads = c->mixed ? kRowBlock : c->row_threads;
  const ImgDesc* imgs = c->L.d_imgs;
  const int2* items = view_list ? c->L.d_rv : c->L.d_row;
  int n = view_list ? c->L.n_rv : c->L.n_row;
  void* args4[] = {(void*)&imgs, (void*)&items, (void*)&n, (void*)&extra};
  return launch_pdl(fn, n, threads, smem, c->s, args4);
}

// Row lists of the hot passes with R rows per item (every problem of a uniform context; a mixed
// context keeps the 256-thread tiles of the multi-size kernels), uploaded with the descriptors.
sgp_status fill_row_items(sgp_ctx* c, int R) {
  Layout& L = c->L;
  c->row.clear();
  c->rv.clear();
  int r0 = 0, rv0 = 0;
  for (int i : c->order) {
    ImgDesc& d = L.d[i];
    const int rpi = c->mixed ? rows_per_item(d.W) : R;
    d.rpi = rpi;
    d.row_item0 = r0;
    d.rv_item0 = rv0;
    d.n_row_items = (d.H + rpi - 1) / rpi;
    d.n_rv_items = d.n_row_items * d.p;
    for (int y = 0; y < d.H; y += rpi) c->row.push_back(make_int2(i, y));
    for (int j = 0; j < d.p; ++j)
      for (int y = 0; y < d.H; y += rpi) c->rv.push_back(make_int2(i, y | (j << 16)));
    r0 += d.n_row_items;
    rv0 += d.n_rv_items;
  }
  if (r0 > L.cap_row || rv0 > L.cap_rv) return fail(SGP_ERR_ARG, "row tile below the planned minimum");
  // view-major copy (uniform contexts: every problem has p views): the items of view j of every
  // problem are the contiguous range [j * n_row, (j + 1) * n_row)
  c->rvo.clear();
  if (!c->mixed)
    for (int j = 0; j < c->p; ++j)
      for (int i : c->order)
        for (int y = 0; y < L.d[i].H; y += L.d[i].rpi) c->rvo.push_back(make_int2(i, y | (j << 16)));
  L.n_row = r0;
  L.n_rv = rv0;
  if (!c->mixed) {
    const int si = side_index(c->W), rm = g_reg.row_rows[si];
    c->rpi_hot = R;
    c->row_threads = R * (kRowBlock / rm);
    c->row_smem_hot = g_reg.row_smem[si] / size_t(rm) * size_t(R);
  }
  // Dry controller runs pay when a pass is one wave of at least one block per SM: every block is
  // resident from the start (a dry run delays no waiting block) and the arrivals spread over
  // microseconds (the early dry runs end before the last block's real one).
  {
    int dev = 0, nsm = 0, occ = 1 << 30;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const RowOp ops[] = {ROP_SGP_UPDATE, ROP_SGP_GRAD, ROP_SGP_AD, ROP_RL_RATIO};
    for (RowOp op : ops)
      for (int f = 0; f < 2; ++f) {
        const void* fn = c->mixed ? g_reg.row_multi[op][f] : g_reg.row[op][f][side_index(c->W)];
        if (!fn) continue;
        int o = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, c->mixed ? kRowBlock : c->row_threads,
                                                         c->mixed ? g_reg.row_multi_smem : c->row_smem_hot));
        occ = std::min(occ, o);
      }
    const int slots = occ == (1 << 30) ? 0 : occ * nsm;
    for (int i = 0; i < c->n; ++i) {
      L.d[i].dry_row = r0 >= nsm && r0 <= slots;
      L.d[i].dry_rv = rv0 >= nsm && rv0 <= slots;
    }
  }
  CU(cudaMemcpyAsync(L.d_imgs, L.d.data(), sizeof(ImgDesc) * c->n, cudaMemcpyHostToDevice, c->s));
  CU(cudaMemcpyAsync(L.d_row, c->row.data(), sizeof(int2) * c->row.size(), cudaMemcpyHostToDevice, c->s));
  CU(cudaMemcpyAsync(L.d_rv, c->rv.data(), sizeof(int2) * c->rv.size(), cudaMemcpyHostToDevice, c->s));
  if (!c->rvo.empty())
    CU(cudaMemcpyAsync(L.d_rvo, c->rvo.data(), sizeof(int2) * c->rvo.size(), cudaMemcpyHostToDevice, c->s));
  CU(cudaStreamSynchronize(c->s));
  return SGP_OK;
}

// jobs are stored job-kind-major: kind k of problem i at index k * n + i; KHAT jobs at 5n + ...
enum JobKind { JOB_A = 0, JOB_AT = 1, JOB_CONJ = 2, JOB_A_RAW = 3, JOB_AT_RAW = 4 };

// variant: COL_1TOP (views list), COL_1TOP_CONJ, COL_PTO1; job_off selects A/AT/CONJ/raw jobs
sgp_status col_pass(sgp_ctx* c, int variant, int job_off, int image = -1) {
  const int si = side_index(image >= 0 ? c->L.d[image].H : c->H);
  int v = variant;
  if (variant == COL_PTO1) v = c->p == 1 ? kColPto1P1 : COL_PTO1;
  const void* fn = g_reg.col[v][si];
  size_t smem = g_reg.col_smem[si];
  if (c->mixed && image < 0) {
    fn = variant == COL_PTO1 ? g_reg.col_multi[c->p == 1 ? 2 : 1] : g_reg.col_multi[0];
    smem = g_reg.col_multi_smem;
  } else if (c->col_narrow && image < 0) {
    fn = g_reg.col_narrow[v];
    smem = g_reg.col_narrow_smem;
  }
  const bool views = variant != COL_PTO1;
  // the iteration's passes (image < 0) run over the PSF band only; a single problem's set-up and
  // operator passes (image >= 0) over every column
  const int2* items = views ? c->L.d_colvb : c->L.d_colb;
  int n = views ? c->L.n_colvb : c->L.n_colb;
  if (image >= 0) {
    items = (views ? c->L.d_colv : c->L.d_col) + (views ? c->colv_begin[image] : c->col_begin[image]);
    n = views ? c->colv_count[image] : c->col_count[image];
  }
  // the job index of an item is the problem index; job_off picks the job kind
  const ColJob* jobs = c->L.d_jobs + job_off;
  void* args[] = {(void*)&jobs, (void*)&items, (void*)&n};
  return launch_pdl(fn, n, kColBlock, smem, c->s, args);
}

// Sum over views of the adjoint column transforms into plane 0 (the column part of
// sum_j A_j^T y_j): one view per item (COL_PTOV) and a view sum for uniform multi-view contexts,
// the single-item form otherwise.
sgp_status adjoint_cols(sgp_ctx* c, int job_off, int image = -1) {
  if (c->p == 1 || c->mixed) return col_pass(c, COL_PTO1, job_off, image);
  sgp_status st = col_pass(c, COL_PTOV, job_off, image);
  if (st) return st;
  const ImgDesc* imgs = c->L.d_imgs;
  int first = image >= 0 ? image : 0, respect = job_off == JOB_AT * c->n ? 1 : 0;
  const int count = image >= 0 ? 1 : c->n;
  const size_t n = size_t(c->H) * c->W / 2;
  const int gx = int(std::min<size_t>((n + 255) / 256, 148 * 4));
  void* a[] = {(void*)&imgs, (void*)&first, (void*)&respect};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(gx, count);
  cfg.blockDim = dim3(256);
  cfg.stream = c->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CU(cudaLaunchKernelExC(&cfg, (const void*)&k_view_sum, a));
  if (g_launch_counter) ++*g_launch_counter;
  return SGP_OK;
}

sgp_status ctrl_pass(sgp_ctx* c, const void* fn) {
  const ImgDesc* imgs = c->L.d_imgs;
  void* args[] = {(void*)&imgs};
  return launch(fn, c->n, kCtrlBlock, 0, c->s, args);
}


sgp_status enter(sgp_ctx* c) {
  g_launch_counter = &c->launches;
  CU(cudaSetDevice(c->device));
  CU(cudaEventRecord(c->ev_in, c->user));
  CU(cudaStreamWaitEvent(c->s, c->ev_in, 0));
  return SGP_OK;
}
sgp_status leave(sgp_ctx* c) {
  g_launch_counter = nullptr;
  CU(cudaEventRecord(c->ev_out, c->s));
  CU(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  return SGP_OK;
}

sgp_status read_ctrl(sgp_ctx* c, CtrlState* dst) {
  CU(cudaMemcpyAsync(dst, c->L.ctrl, sizeof(CtrlState) * c->n, cudaMemcpyDeviceToHost, c->s));
  CU(cudaStreamSynchronize(c->s));
  return SGP_OK;
}

int grid_for(size_t n) { return int(std::min<size_t>((n + 255) / 256, 148 * 16)); }

// plane statistics (see k_stats_partial): out[4 * plane + 0..3]; `scratch` needs 4 * nb * planes doubles
sgp_status plane_stats(cudaStream_t s, const float* x, const float* b, const float* bconst, size_t P, int planes,
                       int mode, double* scratch, double* out) {
  int nb = int(std::min<size_t>(std::max<size_t>(P / 4096, 1), 296));
  void* a1[] = {(void*)&x, (void*)&b, (void*)&bconst, (void*)&P, (void*)&mode, (void*)&scratch};
  CU(cudaLaunchKernel((const void*)&k_stats_partial, dim3(nb, planes), dim3(256), a1, 0, s));
  void* a2[] = {(void*)&scratch, (void*)&nb, (void*)&mode, (void*)&out};
  CU(cudaLaunchKernel((const void*)&k_stats_final, dim3(planes), dim3(256), a2, 0, s));
  return SGP_OK;
}

// ---- iteration sequences --------------------------------------------------------------------------
// kernel launches of one iteration (the launch counter counts graph nodes)
constexpr int kSgpLaunches = 7, kRlLaunches = 4, kFluxLaunches = 2 * (kFluxPasses + 2);

sgp_status seq_rl_unit(sgp_ctx* c) {
  sgp_status st;
  if ((st = row_pass(c, ROP_RL_UPDATE, false))) return st;
  if ((st = col_pass(c, COL_1TOP, JOB_A * c->n))) return st;
  if ((st = row_pass(c, ROP_RL_RATIO, true, 0))) return st;     // + RL controller
  return adjoint_cols(c, JOB_AT * c->n);
}

// One OSEM iteration (Algorithm 2): for j = 0 .. p-1 the sub-step
//   h <- w_{j-1} h A_{j-1}^T r_{j-1}  (pending from the previous sub-step; R2C of h -> plane 0)
//   A_j h -> plane j+1;  r_j - 1 -> plane j+1;  v_j = A_j^T (r_j - 1) in plane j+1
// over the view-major item lists, so that each launch covers view j of every problem: 4p launches
// (the paper's 4p FFTs).  The update of the last view is applied by the next iteration's first
// sub-step, or by the final pass of run_osem.
sgp_status osem_row(sgp_ctx* c, RowOp op, int j, int extra) {
  const void* fn = g_reg.row[op][c->fp64][side_index(c->W)];
  const ImgDesc* imgs = c->L.d_imgs;
  const int2* items = op == ROP_RL_UPDATE ? c->L.d_row : c->L.d_rvo + size_t(j) * c->L.n_row;
  int n = c->L.n_row;
  void* a[] = {(void*)&imgs, (void*)&items, (void*)&n, (void*)&extra};
  return launch_pdl(fn, n, c->row_threads, c->row_smem_hot, c->s, a);
}
sgp_status osem_col(sgp_ctx* c, int variant, int job_off, int j) {
  const int si = side_index(c->H);
  const int2* items = c->L.d_colvo + size_t(j) * c->L.n_colb;
  int n = c->L.n_colb;
  const ColJob* jobs = c->L.d_jobs + job_off;
  void* a[] = {(void*)&jobs, (void*)&items, (void*)&n};
  if (c->col_narrow) return launch_pdl(g_reg.col_narrow[variant], n, kColBlock, g_reg.col_narrow_smem, c->s, a);
  return launch_pdl(g_reg.col[variant][si], n, kColBlock, g_reg.col_smem[si], c->s, a);
}
// PSF band of every problem (after the PSF spectra): cb = 1 + the last spectrum column whose
// entries exceed tol max|K_hat| in some view, rounded up to the column tile; then the column lists
// of the iteration's passes (image < 0) over the band, and the descriptors with cb.
sgp_status apply_band(sgp_ctx* c, const std::vector<int>& raw);
sgp_status set_band(sgp_ctx* c, double tol) {
  Layout& L = c->L;
  std::vector<float> cm;
  std::vector<int> raw(c->n);   // columns in the band before rounding to a column tile
  for (int i = 0; i < c->n; ++i) {
    ImgDesc& d = L.d[i];
    const int M = d.W / 2;
    int cb = M;
    if (tol > 0.0) {
      const float2* kh = reinterpret_cast<const float2*>(L.khat[i]);
      int Hh = d.H, Mm = M, p = d.p;
      float* out = d.u;   // scratch (the iteration state is set later)
      void* a[] = {(void*)&kh, (void*)&Hh, (void*)&Mm, (void*)&p, (void*)&out};
      CU(cudaMemsetAsync(out, 0, sizeof(float) * M, c->s));
      CU(cudaLaunchKernel((const void*)&k_khat_colmax, dim3((M + 127) / 128, std::min(d.H, 64)), dim3(128), a, 0, c->s));
      ++c->launches;
      cm.resize(M);
      CU(cudaMemcpyAsync(cm.data(), out, sizeof(float) * M, cudaMemcpyDeviceToHost, c->s));
      CU(cudaStreamSynchronize(c->s));
      float mx = 0.0f;
      for (float v : cm) mx = std::max(mx, v);
      int last = 0;
      for (int col = 0; col < M; ++col)
        if (cm[col] > float(tol) * mx) last = col;
      cb = last + 1;
    }
    raw[i] = cb;
  }
  // a uniform context of the side with two column plans (16 or 8 values per thread) times both on
  // its own band and keeps the faster (the choice is remembered per size and band for the process)
  if (c->mixed || c->H != kNarrowSide) {
    c->col_narrow = false;
    return apply_band(c, raw);
  }
  static std::map<std::tuple<int, int, int, int>, bool> cache;
  static std::mutex mu;
  const auto key = std::make_tuple(c->H, c->W, c->p, *std::max_element(raw.begin(), raw.end()));
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) {
      c->col_narrow = it->second;
      return apply_band(c, raw);
    }
  }
  // the iteration's two column passes on zeroed planes (the controllers read "running")
  CU(cudaMemsetAsync(L.ctrl, 0, sizeof(CtrlState) * c->n, c->s));
  for (int i = 0; i < c->n; ++i)
    CU(cudaMemsetAsync(L.d[i].spec, 0, sizeof(float) * L.d[i].P * (L.d[i].p + 1), c->s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  sgp_status st = SGP_OK;
  float ms[2] = {1e30f, 1e30f};
  for (int narrow = 0; narrow < 2 && st == SGP_OK; ++narrow) {
    c->col_narrow = narrow != 0;
    if ((st = apply_band(c, raw))) break;
    for (int round = 0; round < 4 && st == SGP_OK; ++round) {   // round 0 warms up
      cudaEventRecord(e0, c->s);
      for (int r = 0; r < 3 && st == SGP_OK; ++r) {
        st = col_pass(c, COL_1TOP, JOB_A * c->n);
        if (st == SGP_OK) st = adjoint_cols(c, JOB_AT * c->n);
      }
      cudaEventRecord(e1, c->s);
      float t = 0.0f;
      if (st == SGP_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = fail(SGP_ERR_CUDA, "column-plan timing failed");
      if (round > 0) ms[narrow] = std::min(ms[narrow], t);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  c->col_narrow = ms[1] < ms[0];
  {
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace(key, c->col_narrow);
  }
  return apply_band(c, raw);
}

// The PSF band rounded to whole column tiles of the chosen plan, the column item lists over it
// and the descriptors with cb.
sgp_status apply_band(sgp_ctx* c, const std::vector<int>& raw) {
  Layout& L = c->L;
  const int cpi_n = g_reg.col_narrow_cols;
  auto tile_of = [&](const ImgDesc& d) { return c->col_narrow ? cpi_n : cols_per_item(d.H); };
  for (int i = 0; i < c->n; ++i) {   // the band rounded up to whole column tiles
    ImgDesc& d = L.d[i];
    const int cpi = tile_of(d);
    d.cb = std::min(d.W / 2, ((raw[i] + cpi - 1) / cpi) * cpi);
  }
  std::vector<int2> vb, b;
  c->colvo.clear();
  for (int i : c->order) {
    const ImgDesc& d = L.d[i];
    const int cpi = tile_of(d);
    for (int j = 0; j < d.p; ++j)
      for (int x = 0; x < d.cb; x += cpi) vb.push_back(make_int2(i, x | (j << 16)));
    for (int x = 0; x < d.cb; x += cpi) b.push_back(make_int2(i, x));
  }
  if (!c->mixed)   // view-major column list of the OSEM sub-steps
    for (int j = 0; j < c->p; ++j)
      for (int i : c->order)
        for (int x = 0; x < L.d[i].cb; x += tile_of(L.d[i])) c->colvo.push_back(make_int2(i, x | (j << 16)));
  if (int(vb.size()) > L.cap_colvb || int(b.size()) > L.cap_colb || int(c->colvo.size()) > L.cap_colvb)
    return fail(SGP_ERR_ARG, "column tile below the planned minimum");
  L.n_colvb = int(vb.size());
  L.n_colb = int(b.size());
  CU(cudaMemcpyAsync(L.d_colvb, vb.data(), sizeof(int2) * vb.size(), cudaMemcpyHostToDevice, c->s));
  CU(cudaMemcpyAsync(L.d_colb, b.data(), sizeof(int2) * b.size(), cudaMemcpyHostToDevice, c->s));
  if (!c->colvo.empty())
    CU(cudaMemcpyAsync(L.d_colvo, c->colvo.data(), sizeof(int2) * c->colvo.size(), cudaMemcpyHostToDevice, c->s));
  CU(cudaMemcpyAsync(L.d_imgs, L.d.data(), sizeof(ImgDesc) * c->n, cudaMemcpyHostToDevice, c->s));
  CU(cudaStreamSynchronize(c->s));
  return SGP_OK;
}

sgp_status seq_osem_iteration(sgp_ctx* c) {
  sgp_status st;
  for (int j = 0; j < c->p; ++j) {
    if ((st = osem_row(c, ROP_RL_UPDATE, j, (j + c->p - 1) % c->p))) return st;
    if ((st = osem_col(c, COL_1TOP, JOB_A * c->n, j))) return st;
    if ((st = osem_row(c, ROP_RL_RATIO, j, 2))) return st;
    if ((st = osem_col(c, COL_PTOV, JOB_AT * c->n, j))) return st;
  }
  return SGP_OK;
}

// flux-constrained projection: bracket, kFluxPasses candidate passes, exact final solve
sgp_status seq_flux(sgp_ctx* c) {
  sgp_status st;
  const bool f = c->fp64;
  const void* fp = f ? (const void*)&k_flux_pass<true> : (const void*)&k_flux_pass<false>;
  const void* fc = f ? (const void*)&k_ctrl_flux<true> : (const void*)&k_ctrl_flux<false>;
  const ImgDesc* imgs = c->L.d_imgs;
  const int2* items = c->L.d_row;
  int n = c->L.n_row;
  for (int step = 0; step < kFluxPasses + 2; ++step) {
    int mode = step == 0 ? 0 : (step <= kFluxPasses ? 1 : 2);
    void* a[] = {(void*)&imgs, (void*)&items, (void*)&n, (void*)&mode};
    if ((st = launch_pdl(fp, n, kRowBlock, 0, c->s, a))) return st;
    void* b[] = {(void*)&imgs, (void*)&mode};
    if ((st = launch_pdl(fc, c->n, kCtrlBlock, 0, c->s, b))) return st;
  }
  return SGP_OK;
}

sgp_status seq_sgp_unit(sgp_ctx* c, bool land = false) {
  sgp_status st;
  if ((st = row_pass(c, ROP_SGP_UPDATE, true))) return st;     // + iteration controller
  if ((st = adjoint_cols(c, JOB_AT * c->n))) return st;
  if ((st = row_pass(c, ROP_SGP_GRAD, false))) return st;      // + step-length controller
  if (c->prm.constraint == 1 && (st = seq_flux(c))) return st;
  if ((st = row_pass(c, ROP_SGP_Y, false))) return st;
  if ((st = col_pass(c, COL_1TOP, JOB_A * c->n))) return st;
  if ((st = row_pass(c, ROP_SGP_AD, true))) return st;         // + line-search controller
  if ((st = row_pass(c, ROP_SGP_ARMX, false))) return st;      // + its continuation
  for (int i = 0; land && i < kLandPasses; ++i)                // landed stop: shorten the last step
    if ((st = row_pass(c, ROP_SGP_LAND, false))) return st;
  return SGP_OK;
}

// a stop decided in the last unit of a graph leaves the update f^(k+1) = f^(k) + lambda d pending
sgp_status seq_sgp_finalize(sgp_ctx* c) { return row_pass(c, ROP_SGP_UPDATE, true); }

sgp_status build_graph(sgp_ctx* c, bool sgp, cudaGraphExec_t* out) {
  if (*out) return SGP_OK;
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
  long long* saved = g_launch_counter;
  g_launch_counter = nullptr;
  sgp_status st = SGP_OK;
  for (int u = 0; u < c->graph_units && st == SGP_OK; ++u) st = sgp ? seq_sgp_unit(c) : seq_rl_unit(c);
  cudaError_t e = cudaStreamEndCapture(c->s, &g);
  g_launch_counter = saved;
  if (st) { if (g) cudaGraphDestroy(g); return st; }
  if (e != cudaSuccess) return fail(SGP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SGP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return SGP_OK;
}

// Fresh controller state for every problem, with the current iterate moved to f[0].
// The solve loop of run_until as one graph: a WHILE node whose body is kLoopUnroll iterations
// (the same passes as a unit of build_graph) followed by k_loop_cond, which ends the loop when
// every problem has stopped or after `cap` bodies.  The iteration count stays on the device, so a
// solve needs no host round trip.  Every pass of an iteration returns at once for a problem that
// has stopped, so an iteration of the body after the stop costs only its launches; two iterations
// per body halve the loop's own cost (the condition kernel and the relaunch of the body).
constexpr int kLoopCounter = 4;   // index of the loop counter in L.d_flag
constexpr int kLoopUnroll = 2;    // iterations per body of the solve loop
sgp_status build_loop_graph(sgp_ctx* c, bool sgp, bool land, int cap, cudaGraphExec_t* out,
                            cudaGraphConditionalHandle* hout) {
  if (*out) return SGP_OK;
  cudaGraph_t g = nullptr;
  CU(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h = 0;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(c->s, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(SGP_ERR_CUDA, std::string("solve loop graph: ") + cudaGetErrorString(e));
  }
  long long* saved = g_launch_counter;
  g_launch_counter = nullptr;
  sgp_status st = SGP_OK;
  for (int u = 0; u < kLoopUnroll && st == SGP_OK; ++u) st = sgp ? seq_sgp_unit(c, land) : seq_rl_unit(c);
  if (st == SGP_OK) {
    const ImgDesc* imgs = c->L.d_imgs;
    int n = c->n, cp = (cap + kLoopUnroll - 1) / kLoopUnroll;
    int* counter = c->L.d_flag + kLoopCounter;
    void* a[] = {(void*)&imgs, (void*)&n, (void*)&h, (void*)&counter, (void*)&cp};
    st = launch_pdl((const void*)&k_loop_cond, 1, 128, 0, c->s, a);
  }
  cudaGraph_t body = nullptr;
  e = cudaStreamEndCapture(c->s, &body);
  g_launch_counter = saved;
  if (st || e != cudaSuccess) {
    cudaGraphDestroy(g);
    return st ? st : fail(SGP_ERR_CUDA, std::string("solve loop capture: ") + cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(SGP_ERR_CUDA, std::string("solve loop instantiate: ") + cudaGetErrorString(e));
  *hout = h;
  return SGP_OK;
}

// Fresh controller states for a new run.  The device state is read back only when some problem
// continues from its last iterate (which of f[0], f[1] holds it); with a new start everywhere (the
// usual solve) the host fills the states and uploads them without waiting for the GPU.
sgp_status reset_ctrl(sgp_ctx* c) {
  CtrlState* h = c->h_ctrl;
  CU(cudaEventSynchronize(c->ev_hctrl));   // the previous upload has read h
  bool all_new = true;
  for (int i = 0; i < c->n; ++i) all_new = all_new && c->start_in_f0[i];
  if (!all_new) {
    CU(cudaMemcpyAsync(h, c->L.ctrl, sizeof(CtrlState) * c->n, cudaMemcpyDeviceToHost, c->s));
    CU(cudaStreamSynchronize(c->s));
  }
  for (int i = 0; i < c->n; ++i) {
    const int cur = c->start_in_f0[i] ? 0 : ((h[i].k - h[i].result_prev) & 1);
    c->start_in_f0[i] = 0;
    if (cur) CU(cudaMemcpyAsync(c->L.d[i].f[0], c->L.d[i].f[1], sizeof(float) * c->L.d[i].P,
                                cudaMemcpyDeviceToDevice, c->s));
    CtrlState z;
    memset(&z, 0, sizeof(z));
    const sgp_params& P = c->prm;
    z.k = 0; z.fresh = 1; z.done = 0; z.status = 0; z.have_v = 0;
    z.trace_cap = P.trace_cap;
    z.stop_kind = STOP_FIXED; z.max_iter = 0;
    z.M_alpha = P.M_alpha; z.warmup = P.warmup_iters; z.max_backtracks = P.max_backtracks;
    z.reg_beta = double(float(P.reg_beta));   // the value the passes use
    z.fp64 = c->fp64; z.constraint = P.constraint;
    z.flux_c = P.flux_c > 0.0 ? P.flux_c : c->c_const[i] * c->nS[i];
    z.alpha = P.alpha0; z.alpha_prev = P.alpha0; z.tau = P.tau1; z.lambda = 1.0;
    z.L1 = P.L1; z.L2 = P.L2;
    z.beta = P.beta; z.theta = P.theta; z.alpha0 = P.alpha0; z.tau1 = P.tau1;
    z.alpha_min = P.alpha_min; z.alpha_max = P.alpha_max;
    z.tol = 0; z.eta = 1.0;
    z.inv_pS = c->nS[i] > 0 ? 1.0 / (double(c->L.d[i].p) * c->nS[i]) : 0.0;
    z.ftrue_norm2 = c->ftrue_n2[i];
    z.rho_prev = INFINITY;
    h[i] = z;
  }
  CU(cudaMemcpyAsync(c->L.ctrl, h, sizeof(CtrlState) * c->n, cudaMemcpyHostToDevice, c->s));
  CU(cudaEventRecord(c->ev_hctrl, c->s));
  return SGP_OK;
}

// Set-up passes from f^(0): A_j f0 (kept in u), J_0, one RL step -> L1/L2 (SGP).  mode 1 SGP, 2 RL.
// Autotuner of the row tile: time two row passes that change no iteration state -- the projection
// pass K4 (pointwise work, R2C, partial sums) and the set-up ratio pass (C2R, KL and ratio, R2C;
// it rewrites A f, which the set-up recomputes) -- for the candidate rows-per-item R = R_max,
// R_max/2, ... (256-thread tiles down to 32-thread ones), going to a smaller tile only while the
// current one gives fewer work items than SMs (more blocks than that only add block scheduling and
// arrival atomics, which these two passes do not show), keep the fastest (a smaller tile must win
// by 5 %; best of three rounds), and remember the choice for the process per (H, W, p), so that
// contexts of one size share it (and their summation order).  It runs before the set-up passes.
sgp_status autotune_rows(sgp_ctx* c) {
  static std::map<std::tuple<int, int, int>, int> cache;
  static std::mutex mu;
  const auto key = std::make_tuple(c->H, c->W, c->p);
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) return fill_row_items(c, it->second);
  }
  const int rmax = rows_per_item(c->W), rmin = rows_min(c->W);
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  sgp_status st = SGP_OK;
  float best = 0.0f;
  int best_r = rmax;
  for (int R = rmax; R >= rmin && st == SGP_OK; R /= 2) {
    if ((st = fill_row_items(c, R))) break;
    if ((st = row_pass(c, ROP_SGP_Y, false))) break;           // warm-up
    if ((st = row_pass(c, ROP_RL_RATIO, true, 1))) break;
    float ms = 1e30f;                                          // best of three rounds
    for (int round = 0; round < 3 && st == SGP_OK; ++round) {
      cudaEventRecord(e0, c->s);
      for (int r = 0; r < 2 && st == SGP_OK; ++r) {
        st = row_pass(c, ROP_SGP_Y, false);
        if (st == SGP_OK) st = row_pass(c, ROP_RL_RATIO, true, 1);
      }
      cudaEventRecord(e1, c->s);
      float t = 0.0f;
      if (st == SGP_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = fail(SGP_ERR_CUDA, "autotuner timing failed");
      ms = std::min(ms, t);
    }
    if (st == SGP_OK && (R == rmax || ms < 0.95f * best)) { best = ms; best_r = R; }
    if (c->L.n_rv >= sms) break;   // this tile already fills every SM: smaller ones only add blocks
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  {
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace(key, best_r);
  }
  return fill_row_items(c, best_r);
}

// report = false (the solve loops): the set-up's status is not read back here; a problem whose
// set-up failed is stopped with its status, which the caller reads after the loop.
sgp_status prepare(sgp_ctx* c, int mode, bool report = true) {
  for (int i = 0; i < c->n; ++i)
    if (!c->has_data[i]) return fail(SGP_ERR_STATE, "sgp_set_data was not called for every problem");
  sgp_status st;
  if ((st = reset_ctrl(c))) return st;
  if (!c->mixed && !c->tuned) {
    c->tuned = true;
    if ((st = autotune_rows(c))) return st;
  }
  if (c->prm.constraint == 1 && mode == 1) {   // flux-constrained start: scale f0 to sum c
    for (int i = 0; i < c->n; ++i) {
      ImgDesc& d = c->L.d[i];
      const double target = c->prm.flux_c > 0.0 ? c->prm.flux_c : c->c_const[i] * c->nS[i];
      if (!(target > 0.0)) return fail(SGP_ERR_ARG, "flux constraint needs a positive flux");
      if ((st = plane_stats(c->s, d.f[0], nullptr, nullptr, d.P, 1, 0, reinterpret_cast<double*>(d.Ad),
                            c->L.scratch[i])))
        return st;
      float* f0 = d.f[0];
      const double* sum = c->L.scratch[i];
      size_t P = d.P;
      double tg = target;
      void* a[] = {(void*)&f0, (void*)&P, (void*)&sum, (void*)&tg};
      if ((st = launch((const void*)&k_scale, grid_for(P), 256, 0, c->s, a))) return st;
    }
  }
  if ((st = row_pass(c, ROP_RL_UPDATE, false))) return st;       // R2C of f0 into plane 0
  if ((st = col_pass(c, COL_1TOP, JOB_A * c->n))) return st;
  if ((st = row_pass(c, ROP_RL_RATIO, true, 1))) return st;      // u = A f0, J_0, r spectra
  if ((st = adjoint_cols(c, JOB_AT * c->n))) return st;    // plane 0 = sum_j A_j^T r_j
  const bool bounds = mode == 1;
  if (bounds && (st = row_pass(c, ROP_MINMAX, false))) return st;
  {
    const ImgDesc* imgs = c->L.d_imgs;
    int adaptive = c->prm.adaptive_L, wb = bounds ? 1 : 0;
    void* args[] = {(void*)&imgs, (void*)&adaptive, (void*)&wb};
    if ((st = launch(c->fp64 ? (const void*)&k_ctrl_setup<true> : (const void*)&k_ctrl_setup<false>, c->n,
                     kCtrlBlock, 0, c->s, args)))
      return st;
  }
  if (mode == 2) {
    // the set-up left sum_j A_j^T r_j of f0 in plane 0: RL continues from there
    for (int i = 0; i < c->n; ++i) {
      int one = 1;
      CU(cudaMemcpyAsync(&c->L.ctrl[i].have_v, &one, sizeof(int), cudaMemcpyHostToDevice, c->s));
      CU(cudaStreamSynchronize(c->s));
    }
  }
  if (!report) {
    c->mode = mode;
    return SGP_OK;
  }
  CU(read_ctrl(c, c->h_ctrl) == SGP_OK ? cudaSuccess : cudaErrorUnknown);
  // a problem whose set-up failed stays stopped with its status; the others proceed
  int failed = 0, first = -1;
  for (int i = 0; i < c->n; ++i)
    if (c->h_ctrl[i].status) { ++failed; if (first < 0) first = i; }
  // the context counts as prepared either way: the state (status, start) stays readable, and a
  // later solve returns the failed problems' status at once, until new data or a new start
  c->mode = mode;
  if (failed == c->n)
    return fail(sgp_status(c->h_ctrl[first].status), "set-up failed for problem " + std::to_string(first) +
                                                         " (no positive pixel after one RL step, or non-finite J)");
  return SGP_OK;
}

sgp_status arm(sgp_ctx* c, int kind, int n_iter, double tol, double eta) {
  const ImgDesc* imgs = c->L.d_imgs;
  int n = c->n, rel = 1;
  void* args[] = {(void*)&imgs, (void*)&n, (void*)&kind, (void*)&n_iter, (void*)&tol, (void*)&eta, (void*)&rel};
  return launch((const void*)&k_ctrl_arm, (n + 127) / 128, 128, 0, c->s, args);
}

sgp_status run_fixed(sgp_ctx* c, bool sgp, int n_iter) {
  if (n_iter < 0) return fail(SGP_ERR_ARG, "negative iteration count");
  sgp_status st;
  if (c->mode != (sgp ? 1 : 2) && (st = prepare(c, sgp ? 1 : 2))) return st;
  if (n_iter == 0) return SGP_OK;
  if ((st = build_graph(c, sgp, sgp ? &c->g_sgp : &c->g_rl))) return st;
  if ((st = arm(c, STOP_FIXED, n_iter, 0.0, 1.0))) return st;
  const int launches = (n_iter + c->graph_units - 1) / c->graph_units;
  for (int l = 0; l < launches; ++l) {
    CU(cudaGraphLaunch(sgp ? c->g_sgp : c->g_rl, c->s));
    const int vs = (c->p > 1 && !c->mixed) ? 1 : 0;
    c->launches += c->graph_units * ((sgp ? (c->prm.constraint == 1 ? kSgpLaunches + kFluxLaunches : kSgpLaunches)
                                          : kRlLaunches) + vs);
  }
  if (sgp && (st = seq_sgp_finalize(c))) return st;
  return SGP_OK;
}

sgp_status run_until(sgp_ctx* c, bool sgp, const sgp_stop_rule* rule, int* iters) {
  if (!rule) return fail(SGP_ERR_ARG, "rule is NULL");
  if (rule->kind < 0 || rule->kind > 4) return fail(SGP_ERR_ARG, "unknown stop rule");
  if (rule->max_iter <= 0) return fail(SGP_ERR_ARG, "max_iter must be positive");
  const bool land = rule->kind == STOP_LANDED;
  if (land && !sgp) return fail(SGP_ERR_ARG, "the landed discrepancy stop is an SGP rule");
  if (land && !(rule->tol < 0.5)) return fail(SGP_ERR_ARG, "landed stop: tol must be below 0.5");
  const double tol = land && rule->tol <= 0.0 ? 1e-5 : rule->tol;
  sgp_status st;
  if (c->mode != (sgp ? 1 : 2) && (st = prepare(c, sgp ? 1 : 2, false))) return st;
  if (rule->kind == STOP_MIN_ERROR)
    for (int i = 0; i < c->n; ++i)
      if (!c->truth[i]) return fail(SGP_ERR_ARG, "minimum-error stop needs sgp_set_truth");
  // one graph launch: a device-side loop of iterations until every problem has stopped (or
  // at least max_iter + 2 iterations, past the controllers' own cap)
  const int cap = rule->max_iter + 2;
  cudaGraphExec_t* gp = land ? &c->gl_land : (sgp ? &c->gl_sgp : &c->gl_rl);
  cudaGraphConditionalHandle* hp = land ? &c->hl_land : (sgp ? &c->hl_sgp : &c->hl_rl);
  if (*gp && c->loop_cap != cap) {   // the cap is a kernel argument of the captured body
    if (c->gl_sgp) { cudaGraphExecDestroy(c->gl_sgp); c->gl_sgp = nullptr; }
    if (c->gl_rl) { cudaGraphExecDestroy(c->gl_rl); c->gl_rl = nullptr; }
    if (c->gl_land) { cudaGraphExecDestroy(c->gl_land); c->gl_land = nullptr; }
  }
  c->loop_cap = cap;
  if ((st = build_loop_graph(c, sgp, land, cap, gp, hp))) return st;
  if ((st = arm(c, rule->kind, rule->max_iter, tol, rule->eta))) return st;
  const int vs = (c->p > 1 && !c->mixed) ? 1 : 0;      // view-sum launch of the adjoint
  const int per_iter = sgp ? (c->prm.constraint == 1 ? kSgpLaunches + kFluxLaunches : kSgpLaunches) +
                                 (land ? kLandPasses : 0) + vs
                           : kRlLaunches + vs;
  const int per_body = kLoopUnroll * per_iter + 1;   // + the loop condition
  CU(cudaMemsetAsync(c->L.d_flag + kLoopCounter, 0, sizeof(int), c->s));
  CU(cudaGraphLaunch(*gp, c->s));
  if (sgp && (st = seq_sgp_finalize(c))) return st;
  int bodies = 0;
  CU(cudaMemcpyAsync(&bodies, c->L.d_flag + kLoopCounter, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  if ((st = read_ctrl(c, c->h_ctrl))) return st;
  c->launches += (long long)bodies * per_body;
  sgp_status res = SGP_OK;
  for (int i = 0; i < c->n; ++i) {
    const CtrlState& h = c->h_ctrl[i];
    if (iters) iters[i] = h.k - h.result_prev;
    if (h.status && res == SGP_OK)
      res = fail(sgp_status(h.status), h.k == 0 ? "set-up failed for problem " + std::to_string(i) +
                                                      " (no positive pixel after one RL step, or non-finite J)"
                                                : "problem " + std::to_string(i) + " stopped with an error");
    if (res == SGP_OK && (h.done < 1 || (rule->kind != STOP_FIXED && h.capped)))
      res = fail(SGP_ERR_TIMEOUT, "problem " + std::to_string(i) + ": stop rule not reached within max_iter");
  }
  return res;
}

// n OSEM iterations from the current iterate; afterwards J_0 of the result (kl_value) and u = A f.
sgp_status run_osem(sgp_ctx* c, int n_iter) {
  if (n_iter < 0) return fail(SGP_ERR_ARG, "negative iteration count");
  if (c->mixed) return fail(SGP_ERR_STATE, "OSEM needs problems of one size");
  sgp_status st;
  if (c->mode != 3) {
    for (int i = 0; i < c->n; ++i)
      if (!c->has_data[i]) return fail(SGP_ERR_STATE, "sgp_set_data was not called for every problem");
    if ((st = reset_ctrl(c))) return st;   // k = 0, no pending update; f[0] holds the start
    if (!c->tuned) {
      c->tuned = true;
      if ((st = autotune_rows(c))) return st;
    }
    c->mode = 3;
  }
  if (n_iter == 0) return SGP_OK;
  if (!c->g_osem) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
    long long* saved = g_launch_counter;
    g_launch_counter = nullptr;
    st = seq_osem_iteration(c);
    cudaError_t e = cudaStreamEndCapture(c->s, &g);
    g_launch_counter = saved;
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return fail(SGP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->g_osem, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(SGP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  for (int l = 0; l < n_iter; ++l) {
    CU(cudaGraphLaunch(c->g_osem, c->s));
    c->launches += 4 * c->p;
  }
  // the pending update of view p-1, then J_0 and u at the result (as in the set-up)
  if ((st = osem_row(c, ROP_RL_UPDATE, 0, c->p - 1))) return st;
  {
    const ImgDesc* imgs = c->L.d_imgs;
    int n = c->n, zero = 0;
    void* a[] = {(void*)&imgs, (void*)&n, (void*)&zero};
    if ((st = launch((const void*)&k_osem_tick, n, 32, 0, c->s, a))) return st;
  }
  if ((st = col_pass(c, COL_1TOP, JOB_A * c->n))) return st;
  if ((st = row_pass(c, ROP_RL_RATIO, true, 1))) return st;
  {
    const ImgDesc* imgs = c->L.d_imgs;
    int adaptive = 0, wb = 0;
    void* args[] = {(void*)&imgs, (void*)&adaptive, (void*)&wb};
    if ((st = launch(c->fp64 ? (const void*)&k_ctrl_setup<true> : (const void*)&k_ctrl_setup<false>, c->n,
                     kCtrlBlock, 0, c->s, args)))
      return st;
  }
  return SGP_OK;
}

sgp_status check_image(sgp_ctx* c, int image) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  if (image < 0 || image >= c->n) return fail(SGP_ERR_ARG, "image index out of range");
  return SGP_OK;
}

}  // namespace

// ================================================================================== C ABI
extern "C" {

void sgp_params_default(sgp_params* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->beta = 1e-4; o->theta = 0.4; o->alpha0 = 1.3; o->tau1 = 0.5;
  o->alpha_min = 1e-5; o->alpha_max = 1e5; o->M_alpha = 3; o->warmup_iters = 20;
  o->adaptive_L = 1; o->max_backtracks = 30; o->L1 = 1e-10; o->L2 = 1e10; o->sigma_R = 1e-2;
  o->constraint = 0; o->flux_c = 0.0; o->reduce_fp64 = 1; o->trace_cap = 4096;
  o->band_tol = 1e-6;
  o->reg_beta = 0.0;
}

const char* sgp_last_error(void) { return g_err.c_str(); }

static sgp_status validate_shapes(int n, const sgp_shape* sh) {
  if (n <= 0 || !sh) return fail(SGP_ERR_ARG, "need at least one problem");
  for (int i = 0; i < n; ++i) {
    if (side_index(sh[i].H) < 0 || side_index(sh[i].W) < 0)
      return fail(SGP_ERR_SIZE_UNSUPPORTED, "H and W must be 16..2048 and a power of two or 3 times one");
    if (sh[i].p < 1 || sh[i].p > kMaxViews) return fail(SGP_ERR_SIZE_UNSUPPORTED, "p must be 1..8");
    if (sh[i].psf_origin != SGP_PSF_CENTER && sh[i].psf_origin != SGP_PSF_CORNER)
      return fail(SGP_ERR_ARG, "psf_origin must be SGP_PSF_CENTER or SGP_PSF_CORNER");
    if (sh[i].p != sh[0].p) return fail(SGP_ERR_SIZE_UNSUPPORTED, "problems of one context must share p");
  }
  return SGP_OK;
}

size_t sgp_workspace_bytes(int n, const sgp_shape* shapes, const sgp_params* params) {
  if (validate_shapes(n, shapes) != SGP_OK) return 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (!g_reg_ready) {
    register_all(g_reg);
    g_reg_ready = true;
  }
  sgp_params P;
  if (params) P = *params; else sgp_params_default(&P);
  std::vector<unsigned char> hb(n, 1);   // count room for background arrays
  Layout L;
  plan_layout(nullptr, n, shapes, std::max(P.trace_cap, 1), reinterpret_cast<const bool*>(hb.data()), L);
  return L.bytes;
}

sgp_status sgp_create_batch(sgp_ctx** out, int n, const sgp_shape* shapes, const sgp_inputs* in,
                            const sgp_params* params, void* workspace, size_t workspace_bytes, void* stream) {
  if (!out) return fail(SGP_ERR_ARG, "out is NULL");
  *out = nullptr;
  sgp_status st = validate_shapes(n, shapes);
  if (st) return st;
  if (!in) return fail(SGP_ERR_ARG, "inputs are NULL");
  if (!workspace) return fail(SGP_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return fail(SGP_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  for (int i = 0; i < n; ++i) {
    if (!in[i].psfs) return fail(SGP_ERR_ARG, "psfs is NULL");
    if (shapes[i].has_mask && !in[i].mask) return fail(SGP_ERR_ARG, "has_mask set but mask is NULL");
  }
  sgp_params P;
  if (params) P = *params; else sgp_params_default(&P);
  if (P.M_alpha < 1 || P.M_alpha > kMaxHist) return fail(SGP_ERR_ARG, "M_alpha must be 1..16");
  if (P.max_backtracks < 0 || P.max_backtracks > 30) return fail(SGP_ERR_ARG, "max_backtracks must be 0..30");
  if (!(P.reg_beta >= 0.0) || !(P.reg_beta < 1e30)) return fail(SGP_ERR_ARG, "reg_beta must be finite and >= 0");
  if (!(P.theta > 0 && P.theta < 1) || !(P.beta > 0 && P.beta < 1)) return fail(SGP_ERR_ARG, "beta, theta must lie in (0,1)");
  if (!(P.alpha_min > 0 && P.alpha_min < P.alpha_max)) return fail(SGP_ERR_ARG, "need 0 < alpha_min < alpha_max");
  if (!P.adaptive_L && !(P.L1 > 0 && P.L1 < P.L2)) return fail(SGP_ERR_ARG, "need 0 < L1 < L2");
  if (P.trace_cap < 1) P.trace_cap = 1;
  if (P.constraint != 0 && P.constraint != 1) return fail(SGP_ERR_ARG, "constraint must be 0 or 1");

  int dev = 0;
  CU(cudaGetDevice(&dev));
  if ((st = ensure_device_ready(dev))) return st;

  sgp_ctx* c = new sgp_ctx();
  c->device = dev;
  c->n = n;
  c->prm = P;
  c->fp64 = P.reduce_fp64 ? 1 : 0;
  c->sh.assign(shapes, shapes + n);
  c->H = shapes[0].H; c->W = shapes[0].W; c->p = shapes[0].p;
  for (int i = 1; i < n; ++i) c->mixed = c->mixed || shapes[i].H != c->H || shapes[i].W != c->W;
  c->user = reinterpret_cast<cudaStream_t>(stream);
  auto bail = [&](sgp_status s) { sgp_destroy(c); return s; };
  if (cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_hctrl, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(SGP_ERR_CUDA, "stream/event creation failed"));
  if (cudaMallocHost(&c->h_ctrl, sizeof(CtrlState) * n) != cudaSuccess)
    return bail(fail(SGP_ERR_CUDA, "pinned host buffer allocation failed"));

  std::vector<unsigned char> hb(n);
  for (int i = 0; i < n; ++i) hb[i] = in[i].b != nullptr;
  plan_layout(nullptr, n, shapes, P.trace_cap, reinterpret_cast<const bool*>(hb.data()), c->L);
  if (c->L.bytes > workspace_bytes)
    return bail(fail(SGP_ERR_WORKSPACE, "workspace too small: need " + std::to_string(c->L.bytes) + " bytes"));
  plan_layout(static_cast<char*>(workspace), n, shapes, P.trace_cap, reinterpret_cast<const bool*>(hb.data()), c->L);
  Layout& L = c->L;
  if ((st = enter(c))) return bail(st);

  // item lists: each problem's items contiguous, problems ordered largest first (the work items of
  // one launch then run longest-first across the SMs)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return L.d[a].P > L.d[b].P; });
  c->order = order;
  c->colv_begin.resize(n); c->colv_count.resize(n); c->col_begin.resize(n); c->col_count.resize(n);
  for (int i : order) {
    ImgDesc& d = L.d[i];
    const int cpi = cols_per_item(d.H), M = d.W / 2;
    c->colv_begin[i] = int(c->colv.size());
    for (int j = 0; j < d.p; ++j)
      for (int x = 0; x < M; x += cpi) c->colv.push_back(make_int2(i, x | (j << 16)));
    c->colv_count[i] = int(c->colv.size()) - c->colv_begin[i];
    c->col_begin[i] = int(c->col.size());
    for (int x = 0; x < M; x += cpi) c->col.push_back(make_int2(i, x));
    c->col_count[i] = int(c->col.size()) - c->col_begin[i];
    d.w_scalar = 1.0f / float(d.p);
    d.a1_scalar = float(d.p);
    d.reg_beta = float(P.reg_beta);
    for (int j = 0; j < kMaxViews; ++j) d.bs[j] = j < d.p ? in[i].b_const[j] : 0.0f;
    d.ftrue = nullptr;
  }
  // column jobs: kinds A, AT, CONJ, A_raw, AT_raw (index kind*n + i), then p KHAT jobs per problem
  c->jobs.assign(L.n_jobs, ColJob{});
  int kh = 5 * n;
  for (int i = 0; i < n; ++i) {
    ImgDesc& d = L.d[i];
    const size_t ps = d.P / 2;
    float2* spec = reinterpret_cast<float2*>(d.spec);
    ColJob base{};
    base.khat = reinterpret_cast<const float2*>(L.khat[i]);
    base.khatq = reinterpret_cast<float2*>(L.khatq[i]);
    base.H = d.H; base.M = d.W / 2; base.plane_stride = ps;
    ColJob a = base;      a.in = spec; a.out = spec + ps; a.nin = 1; a.nout = d.p; a.ctrl = L.ctrl + i;
    ColJob at = base;     at.in = spec + ps; at.out = spec; at.nin = d.p; at.nout = 1; at.ctrl = L.ctrl + i;
    ColJob cj = a;        cj.ctrl = nullptr;
    ColJob ar = a;        ar.ctrl = nullptr;
    ColJob atr = at;      atr.ctrl = nullptr;
    c->jobs[JOB_A * n + i] = a;
    c->jobs[JOB_AT * n + i] = at;
    c->jobs[JOB_CONJ * n + i] = cj;
    c->jobs[JOB_A_RAW * n + i] = ar;
    c->jobs[JOB_AT_RAW * n + i] = atr;
    for (int j = 0; j < d.p; ++j) {
      ColJob k = base;
      k.in = spec + size_t(j + 1) * ps;
      k.out = reinterpret_cast<float2*>(L.khat[i]) + size_t(j) * ps;
      k.khatq = reinterpret_cast<float2*>(L.khatq[i]) + size_t(j) * d.H;
      k.nin = 1; k.nout = 1; k.ctrl = nullptr;
      k.corner = shapes[i].psf_origin == SGP_PSF_CORNER;
      c->jobs[kh++] = k;
    }
  }
  // the column-item lists address job index = problem index; the spectrum set-up needs its own
  std::vector<int> colk_begin(n), colk_count(n);
  for (int i = 0, jb = 5 * n; i < n; ++i) {
    colk_begin[i] = int(c->colk.size());
    const int cpi = cols_per_item(L.d[i].H), M = L.d[i].W / 2;
    for (int j = 0; j < L.d[i].p; ++j, ++jb)
      for (int x = 0; x < M; x += cpi) c->colk.push_back(make_int2(jb, x));
    colk_count[i] = int(c->colk.size()) - colk_begin[i];
  }
  c->c_const.assign(n, 0.0);
  c->nS.assign(n, 0.0);
  c->has_data.assign(n, 0);
  c->truth.assign(n, nullptr);
  c->ftrue_n2.assign(n, 0.0);
  c->start_in_f0.assign(n, 1);

  // PSF statistics and normalisation scale (Sect. 1 / 2.4: unit volume over the domain)
  const size_t P0 = L.d[0].P;
  std::vector<double> stats(4 * kMaxViews);
  for (int i = 0; i < n && st == SGP_OK; ++i) {
    ImgDesc& d = L.d[i];
    if ((st = plane_stats(c->s, in[i].psfs, nullptr, nullptr, d.P, d.p, 0, reinterpret_cast<double*>(d.Ad),
                          L.scratch[i]))) break;
    if (cudaMemcpyAsync(stats.data(), L.scratch[i], sizeof(double) * 4 * d.p, cudaMemcpyDeviceToHost, c->s) != cudaSuccess ||
        cudaStreamSynchronize(c->s) != cudaSuccess) { st = fail(SGP_ERR_CUDA, "PSF statistics failed"); break; }
    for (int j = 0; j < d.p; ++j) {
      const double sum = stats[4 * j], mx = stats[4 * j + 1], mn = stats[4 * j + 2], nf = stats[4 * j + 3];
      if (nf > 0 || !(sum > 0) || !(mx > 0)) { st = fail(SGP_ERR_PSF, "PSF must be finite with a positive sum"); break; }
      if (mn < -1e-6 * mx) { st = fail(SGP_ERR_PSF, "PSF has significantly negative samples"); break; }
      // scale folds the unit-volume normalisation and the 1/(H*M) of the unnormalised transforms;
      // tiny negative round-off is clamped to 0 by the row pass (its effect on the sum is below 1e-6)
      int idx = 5 * n;
      for (int q = 0; q < i; ++q) idx += L.d[q].p;
      c->jobs[idx + j].scale = float(1.0 / (sum * double(d.H) * double(d.W / 2)));
    }
    if (st) break;
    // R2C of each view's PSF into spectrum planes 1..p
    const int si = side_index(d.W);
    const float* src = in[i].psfs;
    float2* dst = reinterpret_cast<float2*>(d.spec) + d.P / 2;
    size_t ivs = d.P, ovs = d.P / 2;
    int Hh = d.H, nv = d.p, clamp = 1;
    const int per_view = (d.H + rows_per_item(d.W) - 1) / rows_per_item(d.W);
    void* a2[] = {(void*)&src, (void*)&ivs, (void*)&dst, (void*)&ovs, (void*)&Hh, (void*)&nv, (void*)&clamp};
    if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view * d.p, kRowBlock, g_reg.row_smem[si], c->s, a2))) break;
  }
  if (st) return bail(st);
  if (cudaMemcpyAsync(L.d_jobs, c->jobs.data(), sizeof(ColJob) * L.n_jobs, cudaMemcpyHostToDevice, c->s) != cudaSuccess ||
      cudaMemcpyAsync(L.d_colv, c->colv.data(), sizeof(int2) * c->colv.size(), cudaMemcpyHostToDevice, c->s) != cudaSuccess ||
      cudaMemcpyAsync(L.d_col, c->col.data(), sizeof(int2) * c->col.size(), cudaMemcpyHostToDevice, c->s) != cudaSuccess ||
      cudaMemcpyAsync(L.d_colk, c->colk.data(), sizeof(int2) * c->colk.size(), cudaMemcpyHostToDevice, c->s) != cudaSuccess)
    return bail(fail(SGP_ERR_CUDA, "descriptor upload failed"));
  if ((st = fill_row_items(c, rows_per_item(c->W)))) return bail(st);
  for (int i = 0; i < n; ++i) {  // PSF spectra (forward column transforms, P/Q packing, scaling, shift)
    const int si = side_index(L.d[i].H);
    const ColJob* jobs = L.d_jobs;
    const int2* items = L.d_colk + colk_begin[i];
    int nk = colk_count[i];
    void* a[] = {(void*)&jobs, (void*)&items, (void*)&nk};
    if ((st = launch(g_reg.col[COL_KHAT][si], nk, kColBlock, g_reg.col_smem[si], c->s, a))) return bail(st);
  }
  if ((st = set_band(c, P.band_tol))) return bail(st);
  for (int i = 0; i < n; ++i) {
    ImgDesc& d = L.d[i];
    if (in[i].b && cudaMemcpyAsync(L.bcopy[i], in[i].b, sizeof(float) * d.P * d.p, cudaMemcpyDeviceToDevice, c->s) != cudaSuccess)
      return bail(fail(SGP_ERR_CUDA, "background copy failed"));
    // zero state so that stray reads are finite
    if (cudaMemsetAsync(d.f[0], 0, sizeof(float) * d.P * 4, c->s) != cudaSuccess)   // f[0], f[1], grad[0], grad[1]
      return bail(fail(SGP_ERR_CUDA, "memset failed"));
  }
  // boundary problems: alpha_j = K_j (x) M_S, R and M_R / alpha (Sect. 2.4, Eq. Rdef)
  for (int i = 0; i < n; ++i) {
    ImgDesc& d = L.d[i];
    if (!d.boundary) continue;
    if (cudaMemcpyAsync(L.mS[i], in[i].mask, d.P, cudaMemcpyDeviceToDevice, c->s) != cudaSuccess)
      return bail(fail(SGP_ERR_CUDA, "mask copy failed"));
    float* mf = d.u;   // scratch plane
    void* a[] = {(void*)&in[i].mask, (void*)&mf, (void*)&d.P};
    if ((st = launch((const void*)&k_u8_to_float, grid_for(d.P), 256, 0, c->s, a))) return bail(st);
    const int si = side_index(d.W);
    float2* sp0 = reinterpret_cast<float2*>(d.spec);
    size_t ivs = d.P, ovs = d.P / 2;
    int Hh = d.H, one = 1, clamp = 0;
    const int per_view = (d.H + rows_per_item(d.W) - 1) / rows_per_item(d.W);
    const float* mfc = mf;
    void* a2[] = {(void*)&mfc, (void*)&ivs, (void*)&sp0, (void*)&ovs, (void*)&Hh, (void*)&one, (void*)&clamp};
    if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view, kRowBlock, g_reg.row_smem[si], c->s, a2))) return bail(st);
    if ((st = col_pass(c, COL_1TOP_CONJ, JOB_CONJ * n, i))) return bail(st);
    const float2* sp1 = sp0 + d.P / 2;
    float* alpha = d.Ad;
    int nv = d.p;
    float sc = 1.0f;
    void* a3[] = {(void*)&sp1, (void*)&ovs, (void*)&alpha, (void*)&ivs, (void*)&Hh, (void*)&nv, (void*)&sc};
    if ((st = launch(g_reg.row[ROP_C2R][0][si], per_view * d.p, kRowBlock, g_reg.row_smem[si], c->s, a3))) return bail(st);
    float sig = float(P.sigma_R);
    float* w = const_cast<float*>(d.w);
    float* wv = const_cast<float*>(d.wv);
    const float* al = alpha;
    void* a4[] = {(void*)&al, (void*)&nv, (void*)&d.P, (void*)&sig, (void*)&w, (void*)&wv};
    if ((st = launch((const void*)&k_make_w, grid_for(d.P), 256, 0, c->s, a4))) return bail(st);
  }
  // controller array: zero, then fresh state at first use
  if (cudaMemsetAsync(L.ctrl, 0, sizeof(CtrlState) * n, c->s) != cudaSuccess) return bail(fail(SGP_ERR_CUDA, "memset failed"));
  if (cudaStreamSynchronize(c->s) != cudaSuccess) {
    return bail(fail(SGP_ERR_CUDA, std::string("set-up kernels failed: ") + cudaGetErrorString(cudaGetLastError())));
  }
  (void)P0;
  if ((st = leave(c))) return bail(st);
  *out = c;
  return SGP_OK;
}

sgp_status sgp_create(sgp_ctx** out, const sgp_shape* shape, const float* psfs, const float* b,
                      const float* b_const, const uint8_t* mask, const sgp_params* params,
                      void* workspace, size_t workspace_bytes, void* stream) {
  if (!shape) return fail(SGP_ERR_ARG, "shape is NULL");
  sgp_status st0 = validate_shapes(1, shape);
  if (st0) return st0;
  sgp_inputs in;
  memset(&in, 0, sizeof(in));
  in.psfs = psfs;
  in.b = b;
  in.mask = mask;
  if (!b) {
    if (!b_const) return fail(SGP_ERR_ARG, "give either a background array or constants");
    for (int j = 0; j < shape->p && j < kMaxViews; ++j) in.b_const[j] = b_const[j];
  }
  return sgp_create_batch(out, 1, shape, &in, params, workspace, workspace_bytes, stream);
}

sgp_status sgp_set_data(sgp_ctx* c, int image, const float* g) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!g) return fail(SGP_ERR_ARG, "g is NULL");
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  int* bad = c->L.d_flag;
  CU(cudaMemsetAsync(bad, 0, sizeof(int), c->s));
  const uint8_t* mask = c->L.mS[image];
  size_t P = d.P;
  int p = d.p;
  {
    float* gout = d.g;
    void* a[] = {(void*)&g, (void*)&mask, (void*)&gout, (void*)&P, (void*)&p, (void*)&bad};
    if ((st = launch((const void*)&k_prepare_data, grid_for(P * p), 256, 0, c->s, a))) return st;
  }
  {
    float* bc = reinterpret_cast<float*>(c->L.scratch[image] + 56);   // p floats of constants
    CU(cudaMemcpyAsync(bc, d.bs, sizeof(float) * kMaxViews, cudaMemcpyHostToDevice, c->s));
    if ((st = plane_stats(c->s, d.g, d.b, bc, P, p, 1, reinterpret_cast<double*>(d.Ad), c->L.scratch[image])))
      return st;
  }
  int hbad = 0;
  double st4[4 * kMaxViews], sums[3 * kMaxViews];
  CU(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CU(cudaMemcpyAsync(st4, c->L.scratch[image], sizeof(double) * 4 * p, cudaMemcpyDeviceToHost, c->s));
  CU(cudaStreamSynchronize(c->s));
  if (hbad) return fail(SGP_ERR_NONFINITE, "data contain negative or non-finite values");
  for (int j = 0; j < p; ++j)
    for (int q = 0; q < 3; ++q) sums[3 * j + q] = st4[4 * j + q];
  // constant start of Sect. 3.1: mean over views of (sum_S g - sum_S b) / |S|
  double cm = 0.0, gm = 0.0;
  const double nS = sums[2];
  if (!(nS > 0)) return fail(SGP_ERR_ARG, "the mask selects no pixel");
  for (int j = 0; j < p; ++j) { cm += (sums[3 * j] - sums[3 * j + 1]) / nS; gm += sums[3 * j] / nS; }
  cm /= p; gm /= p;
  if (!(cm > 0)) cm = std::max(gm, 1e-3);
  c->c_const[image] = cm;
  c->nS[image] = nS;
  c->has_data[image] = 1;
  {
    float* f0 = d.f[0];
    const float* w = d.w;
    const float* src = nullptr;
    float v = float(cm);
    void* a[] = {(void*)&f0, (void*)&w, (void*)&src, (void*)&v, (void*)&P};
    if ((st = launch((const void*)&k_fill_start, grid_for(P), 256, 0, c->s, a))) return st;
  }
  c->start_in_f0[image] = 1;
  c->mode = 0;
  return leave(c);
}

sgp_status sgp_set_start(sgp_ctx* c, int image, int mode, const float* f0) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!c->has_data[image]) return fail(SGP_ERR_STATE, "call sgp_set_data first");
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  float* dst = d.f[0];
  const float* w = d.w;
  const float* src = nullptr;
  float v = 0.0f;
  switch (mode) {
    case SGP_START_ZERO: v = 0.0f; break;
    case SGP_START_DATA: src = d.g; break;   // g_1; pixels outside S carry -1 and clip to 0
    case SGP_START_CONSTANT: v = float(c->c_const[image]); break;
    case SGP_START_USER:
      if (!f0) return fail(SGP_ERR_ARG, "f0 is NULL");
      src = f0;
      break;
    default: return fail(SGP_ERR_ARG, "unknown start mode");
  }
  size_t P = d.P;
  void* a[] = {(void*)&dst, (void*)&w, (void*)&src, (void*)&v, (void*)&P};
  if ((st = launch((const void*)&k_fill_start, grid_for(P), 256, 0, c->s, a))) return st;
  c->start_in_f0[image] = 1;
  c->mode = 0;
  return leave(c);   // stream-ordered: the next call (or the caller's stream) sees f[0]
}

sgp_status sgp_set_truth(sgp_ctx* c, int image, const float* f_true) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  c->truth[image] = f_true;
  d.ftrue = f_true;
  CU(cudaMemcpyAsync(c->L.d_imgs + image, &d, sizeof(ImgDesc), cudaMemcpyHostToDevice, c->s));
  double nrm = 0.0;
  if (f_true) {
    double* out = c->L.scratch[image] + 40;
    size_t P = d.P;
    void* a[] = {(void*)&f_true, (void*)&P, (void*)&out};
    if ((st = launch((const void*)&k_sumsq, 1, 256, 0, c->s, a))) return st;
    CU(cudaMemcpyAsync(&nrm, out, sizeof(double), cudaMemcpyDeviceToHost, c->s));
  }
  CU(cudaMemcpyAsync(&c->L.ctrl[image].ftrue_norm2, &nrm, sizeof(double), cudaMemcpyHostToDevice, c->s));
  CU(cudaStreamSynchronize(c->s));
  c->ftrue_n2[image] = nrm;
  return leave(c);
}

sgp_status rl_iterate(sgp_ctx* c, int n) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  if (c->prm.reg_beta > 0.0) return fail(SGP_ERR_ARG, "reg_beta applies to SGP only");
  sgp_status st = enter(c);
  if (st || (st = run_fixed(c, false, n))) return st;
  return leave(c);
}

sgp_status osem_iterate(sgp_ctx* c, int n) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  if (c->prm.reg_beta > 0.0) return fail(SGP_ERR_ARG, "reg_beta applies to SGP only");
  sgp_status st = enter(c);
  if (st || (st = run_osem(c, n))) return st;
  return leave(c);
}

sgp_status sgp_iterate(sgp_ctx* c, int n) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  sgp_status st = enter(c);
  if (st || (st = run_fixed(c, true, n))) return st;
  return leave(c);
}

sgp_status sgp_solve_until(sgp_ctx* c, const sgp_stop_rule* rule, int* iters) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  sgp_status st = enter(c);
  if (st) return st;
  const sgp_status res = run_until(c, true, rule, iters);
  if ((st = leave(c))) return st;
  return res;
}

sgp_status rl_solve_until(sgp_ctx* c, const sgp_stop_rule* rule, int* iters) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  if (c->prm.reg_beta > 0.0) return fail(SGP_ERR_ARG, "reg_beta applies to SGP only");
  sgp_status st = enter(c);
  if (st) return st;
  const sgp_status res = run_until(c, false, rule, iters);
  if ((st = leave(c))) return st;
  return res;
}

sgp_status sgp_get_info(sgp_ctx* c, int image, sgp_info* o) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!o) return fail(SGP_ERR_ARG, "out is NULL");
  if ((st = enter(c))) return st;
  if (c->mode == 0 && (st = prepare(c, 1))) return st;
  CtrlState h;
  CU(cudaMemcpyAsync(&h, c->L.ctrl + image, sizeof(CtrlState), cudaMemcpyDeviceToHost, c->s));
  CU(cudaStreamSynchronize(c->s));
  memset(o, 0, sizeof(*o));
  o->k = h.k - h.result_prev;
  o->status = h.status;
  o->stopped = h.done >= 1 && !(h.capped && h.stop_kind != STOP_FIXED);
  o->trace_n = h.trace_n;
  o->J = h.J;
  o->D = 2.0 * h.J * h.inv_pS;
  o->L1 = h.L1; o->L2 = h.L2; o->alpha = h.alpha; o->tau = h.tau; o->lambda = h.lambda; o->rho = h.rho;
  o->nS = c->nS[image];
  o->flux_c = c->c_const[image];
  o->band_cols = c->L.d[image].cb;
  o->reg = h.R;
  return leave(c);
}

sgp_status kl_value(sgp_ctx* c, int image, double* out) {
  if (!out) return fail(SGP_ERR_ARG, "out is NULL");
  sgp_info info;
  sgp_status st = sgp_get_info(c, image, &info);
  if (st) return st;
  *out = info.J;
  return SGP_OK;
}

sgp_status sgp_get_f(sgp_ctx* c, int image, float* dst) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!dst) return fail(SGP_ERR_ARG, "dst is NULL");
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  int par = 0;
  if (!c->start_in_f0[image]) {
    CtrlState h;
    CU(cudaMemcpyAsync(&h, c->L.ctrl + image, sizeof(CtrlState), cudaMemcpyDeviceToHost, c->s));
    CU(cudaStreamSynchronize(c->s));
    par = (h.k - h.result_prev) & 1;
  }
  CU(cudaMemcpyAsync(dst, d.f[par], sizeof(float) * d.P, cudaMemcpyDeviceToDevice, c->s));
  CU(cudaStreamSynchronize(c->s));
  return leave(c);
}

sgp_status sgp_get_trace(sgp_ctx* c, int image, double* out, int cap, int* count) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if ((st = enter(c))) return st;
  CtrlState h;
  CU(cudaMemcpyAsync(&h, c->L.ctrl + image, sizeof(CtrlState), cudaMemcpyDeviceToHost, c->s));
  CU(cudaStreamSynchronize(c->s));
  const int avail = std::min(h.trace_n, h.trace_cap);
  const int m = out ? std::min(avail, cap) : 0;
  if (m > 0) {
    CU(cudaMemcpyAsync(out, c->L.d[image].trace, sizeof(double) * kTraceStride * m, cudaMemcpyDeviceToHost, c->s));
    CU(cudaStreamSynchronize(c->s));
  }
  if (count) *count = avail;
  return leave(c);
}

sgp_status sgp_apply_A(sgp_ctx* c, int image, const float* f, float* out) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!f || !out) return fail(SGP_ERR_ARG, "NULL array");
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  const int si = side_index(d.W);
  const int per_view = (d.H + rows_per_item(d.W) - 1) / rows_per_item(d.W);
  size_t P = d.P, ivs = d.P, ovs = d.P / 2;
  int Hh = d.H, one = 1, clamp = 0, p = d.p;
  const float* src = f;
  if (d.boundary) {   // M_R f (into a scratch plane)
    CU(cudaMemcpyAsync(d.Ad, f, sizeof(float) * P, cudaMemcpyDeviceToDevice, c->s));
    float* x = d.Ad;
    const float* w = d.w;
    const float* gnull = nullptr;
    void* a[] = {(void*)&x, (void*)&P, (void*)&one, (void*)&w, (void*)&gnull};
    if ((st = launch((const void*)&k_apply_mask, grid_for(P), 256, 0, c->s, a))) return st;
    src = d.Ad;
  }
  float2* sp0 = reinterpret_cast<float2*>(d.spec);
  void* a2[] = {(void*)&src, (void*)&ivs, (void*)&sp0, (void*)&ovs, (void*)&Hh, (void*)&one, (void*)&clamp};
  if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view, kRowBlock, g_reg.row_smem[si], c->s, a2))) return st;
  if ((st = col_pass(c, COL_1TOP, JOB_A_RAW * c->n, image))) return st;
  const float2* sp1 = sp0 + P / 2;
  float sc = 1.0f;
  void* a3[] = {(void*)&sp1, (void*)&ovs, (void*)&out, (void*)&ivs, (void*)&Hh, (void*)&p, (void*)&sc};
  if ((st = launch(g_reg.row[ROP_C2R][0][si], per_view * p, kRowBlock, g_reg.row_smem[si], c->s, a3))) return st;
  if (d.boundary) {   // M_S (A f)
    const float* wnull = nullptr;
    const float* gg = d.g;   // sentinel -1 outside S, per view
    void* a[] = {(void*)&out, (void*)&P, (void*)&p, (void*)&wnull, (void*)&gg};
    if ((st = launch((const void*)&k_apply_mask, grid_for(P * p), 256, 0, c->s, a))) return st;
  }
  c->mode = 0;
  return leave(c);
}

sgp_status sgp_apply_AT(sgp_ctx* c, int image, const float* y, float* out) {
  sgp_status st = check_image(c, image);
  if (st) return st;
  if (!y || !out) return fail(SGP_ERR_ARG, "NULL array");
  if ((st = enter(c))) return st;
  ImgDesc& d = c->L.d[image];
  const int si = side_index(d.W);
  const int per_view = (d.H + rows_per_item(d.W) - 1) / rows_per_item(d.W);
  size_t P = d.P, ivs = d.P, ovs = d.P / 2;
  int Hh = d.H, one = 1, clamp = 0, p = d.p;
  const float* src = y;
  if (d.boundary) {   // M_S y_j
    CU(cudaMemcpyAsync(d.Ad, y, sizeof(float) * P * p, cudaMemcpyDeviceToDevice, c->s));
    float* x = d.Ad;
    const float* wnull = nullptr;
    const float* gg = d.g;
    void* a[] = {(void*)&x, (void*)&P, (void*)&p, (void*)&wnull, (void*)&gg};
    if ((st = launch((const void*)&k_apply_mask, grid_for(P * p), 256, 0, c->s, a))) return st;
    src = d.Ad;
  }
  float2* sp1 = reinterpret_cast<float2*>(d.spec) + P / 2;
  void* a2[] = {(void*)&src, (void*)&ivs, (void*)&sp1, (void*)&ovs, (void*)&Hh, (void*)&p, (void*)&clamp};
  if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view * p, kRowBlock, g_reg.row_smem[si], c->s, a2))) return st;
  if ((st = adjoint_cols(c, JOB_AT_RAW * c->n, image))) return st;
  const float2* sp0 = reinterpret_cast<const float2*>(d.spec);
  float sc = 1.0f;
  void* a3[] = {(void*)&sp0, (void*)&ovs, (void*)&out, (void*)&ivs, (void*)&Hh, (void*)&one, (void*)&sc};
  if ((st = launch(g_reg.row[ROP_C2R][0][si], per_view, kRowBlock, g_reg.row_smem[si], c->s, a3))) return st;
  if (d.boundary) {   // M_R (...)
    const float* w = d.w;
    const float* gnull = nullptr;
    void* a[] = {(void*)&out, (void*)&P, (void*)&one, (void*)&w, (void*)&gnull};
    if ((st = launch((const void*)&k_apply_mask, grid_for(P), 256, 0, c->s, a))) return st;
  }
  c->mode = 0;
  return leave(c);
}

sgp_status sgp_time_passes(sgp_ctx* c, int iters, double* ms_out, int n_out) {
  if (!c || !ms_out || n_out < kSgpLaunches || iters <= 0)
    return fail(SGP_ERR_ARG, "need ctx, iters > 0 and 7 outputs");
  if (c->prm.constraint != 0) return fail(SGP_ERR_ARG, "pass timing covers the non-negativity constraint only");
  sgp_status st = enter(c);
  if (st) return st;
  if (c->mode != 1 && (st = prepare(c, 1))) return st;
  if ((st = arm(c, STOP_FIXED, 1 << 30, 0.0, 1.0))) return st;
  // every iteration's passes are queued before the host waits once, so the GPU does not idle
  // between iterations (an event pair around each pass; a pass's time includes its launch)
  std::vector<cudaEvent_t> ev(size_t(iters) * (kSgpLaunches + 1));
  for (auto& e : ev) CU(cudaEventCreate(&e));
  std::vector<double> acc(kSgpLaunches, 0.0);
  for (int it = 0; it < iters && st == SGP_OK; ++it) {
    cudaEvent_t* e = ev.data() + size_t(it) * (kSgpLaunches + 1);
    int q = 0;
    CU(cudaEventRecord(e[q++], c->s));
    auto step = [&](sgp_status s2) { if (!st) st = s2; cudaEventRecord(e[q++], c->s); };
    step(row_pass(c, ROP_SGP_UPDATE, true));
    step(adjoint_cols(c, JOB_AT * c->n));
    step(row_pass(c, ROP_SGP_GRAD, false));
    step(row_pass(c, ROP_SGP_Y, false));
    step(col_pass(c, COL_1TOP, JOB_A * c->n));
    step(row_pass(c, ROP_SGP_AD, true));
    step(row_pass(c, ROP_SGP_ARMX, false));
  }
  if (st == SGP_OK && cudaEventSynchronize(ev.back()) != cudaSuccess) st = fail(SGP_ERR_CUDA, "pass timing failed");
  for (int it = 0; it < iters && st == SGP_OK; ++it) {
    cudaEvent_t* e = ev.data() + size_t(it) * (kSgpLaunches + 1);
    for (int k = 0; k < kSgpLaunches; ++k) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, e[k], e[k + 1]) != cudaSuccess) st = fail(SGP_ERR_CUDA, "pass timing failed");
      acc[k] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st) return st;
  for (int k = 0; k < kSgpLaunches; ++k) ms_out[k] = acc[k] / iters;
  c->mode = 0;   // the timed iterations advanced the state; the next solve re-initialises
  return leave(c);
}

long long sgp_launch_count(sgp_ctx* c) { return c ? c->launches : 0; }

sgp_status sgp_get_tile(sgp_ctx* c, int* rows_per_item_out, int* threads_out) {
  if (!c || !rows_per_item_out || !threads_out) return fail(SGP_ERR_ARG, "NULL argument");
  *rows_per_item_out = c->mixed ? 0 : c->rpi_hot;
  *threads_out = c->mixed ? kRowBlock : c->row_threads;
  return SGP_OK;
}

sgp_status sgp_set_tile(sgp_ctx* c, int rows) {
  if (!c) return fail(SGP_ERR_ARG, "ctx is NULL");
  if (c->mixed) return fail(SGP_ERR_STATE, "contexts of mixed sizes keep the multi-size tiles");
  const int rmax = rows_per_item(c->W), rmin = rows_min(c->W);
  bool ok = false;
  for (int R = rmax; R >= rmin; R /= 2) ok = ok || R == rows;
  if (!ok) return fail(SGP_ERR_ARG, "rows per item must be R_max / 2^k with at least 32 threads per block");
  sgp_status st = enter(c);
  if (st) return st;
  CU(cudaStreamSynchronize(c->s));
  // captured graphs hold the old launch geometry
  if (c->g_sgp) { cudaGraphExecDestroy(c->g_sgp); c->g_sgp = nullptr; }
  if (c->g_rl) { cudaGraphExecDestroy(c->g_rl); c->g_rl = nullptr; }
  if (c->g_osem) { cudaGraphExecDestroy(c->g_osem); c->g_osem = nullptr; }
  if (c->gl_sgp) { cudaGraphExecDestroy(c->gl_sgp); c->gl_sgp = nullptr; }
  if (c->gl_rl) { cudaGraphExecDestroy(c->gl_rl); c->gl_rl = nullptr; }
  if (c->gl_land) { cudaGraphExecDestroy(c->gl_land); c->gl_land = nullptr; }
  if ((st = fill_row_items(c, rows))) return st;
  c->tuned = true;
  c->mode = 0;   // the next solve re-initialises the iteration from the current iterate
  return leave(c);
}

// ------------------------------------------------------------------------------ mosaic
static sgp_status mosaic_geom(const sgp_mosaic* m, MosaicGeom& g) {
  if (!m) return fail(SGP_ERR_ARG, "mosaic is NULL");
  if (m->H < 1 || m->W < 1 || m->ny < 1 || m->nx < 1 || m->ny > kMosaicMax || m->nx > kMosaicMax)
    return fail(SGP_ERR_ARG, "mosaic: need H, W >= 1 and 1 <= ny, nx <= 16");
  if (m->sub_h < 1 || m->sub_w < 1 || m->sub_h > m->H || m->sub_w > m->W || m->ext_h < m->sub_h || m->ext_w < m->sub_w)
    return fail(SGP_ERR_ARG, "mosaic: need 1 <= sub <= image and sub <= ext");
  memset(&g, 0, sizeof(g));
  g.H = m->H; g.W = m->W; g.ny = m->ny; g.nx = m->nx; g.sy = m->sub_h; g.sx = m->sub_w;
  g.EH = m->ext_h; g.EW = m->ext_w; g.ey = (m->ext_h - m->sub_h) / 2; g.ex = (m->ext_w - m->sub_w) / 2;
  for (int axis = 0; axis < 2; ++axis) {
    const int N = axis ? m->W : m->H, n = axis ? m->nx : m->ny, sz = axis ? m->sub_w : m->sub_h;
    int* w = axis ? g.wx : g.wy;
    int* cb = axis ? g.cx : g.cy;
    for (int k = 0; k < n; ++k) {
      w[k] = n == 1 ? 0 : int((long long)k * (N - sz) / (n - 1));
      cb[k] = int((long long)k * N / n);
    }
    cb[n] = N;
    for (int k = 0; k < n; ++k)
      if (cb[k] < w[k] || cb[k + 1] > w[k] + sz)
        return fail(SGP_ERR_ARG, "mosaic: a piece is not inside its sub-domain (sub-domains too small)");
  }
  return SGP_OK;
}

sgp_status sgp_mosaic_geometry(const sgp_mosaic* m, int* out) {
  MosaicGeom g;
  sgp_status st = mosaic_geom(m, g);
  if (st || !out) return st;
  int o = 0;
  for (int k = 0; k < g.ny; ++k) { out[o++] = g.wy[k]; out[o++] = g.wy[k] + g.sy; out[o++] = g.cy[k]; out[o++] = g.cy[k + 1]; }
  for (int k = 0; k < g.nx; ++k) { out[o++] = g.wx[k]; out[o++] = g.wx[k] + g.sx; out[o++] = g.cx[k]; out[o++] = g.cx[k + 1]; }
  return SGP_OK;
}

sgp_status sgp_mosaic_split(const sgp_mosaic* m, int p, const float* g, float* tiles, uint8_t* masks, void* stream) {
  MosaicGeom geo;
  sgp_status st = mosaic_geom(m, geo);
  if (st) return st;
  if (p < 1 || p > kMaxViews) return fail(SGP_ERR_SIZE_UNSUPPORTED, "1 <= p <= 8 views");
  if (!g || !tiles || !masks) return fail(SGP_ERR_ARG, "NULL array");
  const size_t total = size_t(geo.EH) * geo.EW * p * geo.ny * geo.nx;
  const int grid = int(std::min<size_t>((total + 255) / 256, 148 * 8));
  k_mosaic_split<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(g, p, geo, tiles, masks);
  CU(cudaGetLastError());
  return SGP_OK;
}

sgp_status sgp_mosaic_stitch(const sgp_mosaic* m, const float* recs, float* f, void* stream) {
  MosaicGeom geo;
  sgp_status st = mosaic_geom(m, geo);
  if (st) return st;
  if (!recs || !f) return fail(SGP_ERR_ARG, "NULL array");
  const size_t total = size_t(geo.H) * geo.W;
  const int grid = int(std::min<size_t>((total + 255) / 256, 148 * 8));
  k_mosaic_stitch<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(recs, geo, f);
  CU(cudaGetLastError());
  return SGP_OK;
}

size_t sgp_sum_terms_workspace_bytes(size_t n) {
  const size_t blocks = (n + size_t(kRowBlock) * kSumPerThread - 1) / (size_t(kRowBlock) * kSumPerThread);
  return 2048 + std::max<size_t>(blocks, 1) * kPartStride * sizeof(double);
}

sgp_status sgp_sum_terms(int kind, int reduce_fp64, const float* a, const float* b, const float* c, size_t n,
                         double lambda, float* terms, double* out, void* workspace, size_t ws_bytes, void* stream) {
  if (!out || !a || n == 0) return fail(SGP_ERR_ARG, "out and a must be non-NULL and n positive");
  if (kind < SGP_SUM_VALUES || kind > SGP_SUM_BB3) return fail(SGP_ERR_ARG, "unknown term kind");
  if ((kind == SGP_SUM_KL || kind >= SGP_SUM_ARMIJO) && !b) return fail(SGP_ERR_ARG, "b is NULL");
  if (kind >= SGP_SUM_ARMIJO && !c) return fail(SGP_ERR_ARG, "c is NULL");
  const size_t per_block = size_t(kRowBlock) * kSumPerThread;
  const size_t blocks = (n + per_block - 1) / per_block;
  if (blocks > size_t(1) << 30) return fail(SGP_ERR_SIZE_UNSUPPORTED, "too many terms");
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || ws_bytes < sgp_sum_terms_workspace_bytes(n))
    return fail(SGP_ERR_WORKSPACE, "workspace missing, misaligned or smaller than sgp_sum_terms_workspace_bytes(n)");
  g_launch_counter = nullptr;   // no context is driven by this call
  int dev = 0;
  CU(cudaGetDevice(&dev));
  sgp_status st = ensure_device_ready(dev);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  CtrlState* cs = reinterpret_cast<CtrlState*>(w);
  double* dout = reinterpret_cast<double*>(w + 1024);
  double* part = reinterpret_cast<double*>(w + 2048);
  static_assert(sizeof(CtrlState) <= 1024, "controller record larger than its slot");
  CU(cudaMemsetAsync(cs, 0, sizeof(CtrlState), s));
  int nb = int(blocks);
  float lam = float(lambda);
  void* args[] = {(void*)&kind, (void*)&a, (void*)&b, (void*)&c, (void*)&n, (void*)&lam, (void*)&terms,
                  (void*)&part, (void*)&cs, (void*)&nb, (void*)&dout};
  const void* fn = reduce_fp64 ? (const void*)&k_sum_terms<true> : (const void*)&k_sum_terms<false>;
  if ((st = launch(fn, nb, kRowBlock, 0, s, args))) return st;
  CU(cudaMemcpyAsync(out, dout, sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return SGP_OK;
}

sgp_status sgp_destroy(sgp_ctx* c) {
  if (!c) return SGP_OK;
  if (g_launch_counter == &c->launches) g_launch_counter = nullptr;
  if (c->s) cudaStreamSynchronize(c->s);
  if (c->g_sgp) cudaGraphExecDestroy(c->g_sgp);
  if (c->g_rl) cudaGraphExecDestroy(c->g_rl);
  if (c->g_osem) cudaGraphExecDestroy(c->g_osem);
  if (c->gl_sgp) cudaGraphExecDestroy(c->gl_sgp);
  if (c->gl_rl) cudaGraphExecDestroy(c->gl_rl);
  if (c->gl_land) cudaGraphExecDestroy(c->gl_land);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->ev_hctrl) cudaEventDestroy(c->ev_hctrl);
  if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
  if (c->s) cudaStreamDestroy(c->s);
  delete c;
  return SGP_OK;
}

}  // extern "C"

// ================================================================================== no-allocation variant
// A periodic single-view convolution whose scratch lives in a fixed device array instead of a
// caller-provided workspace, for callers that cannot allocate device memory.
namespace {

constexpr size_t kNoAllocMaxPixels = 512 * 512;   // H * W limit of sgp_convolve_noalloc
// layout (floats): PSF spectrum P | Q column 2*2048 | spectrum planes 0, 1: 2P | statistics | jobs | items
constexpr size_t kNoAllocStatsOff = 3 * kNoAllocMaxPixels + 4 * 2048;
constexpr size_t kNoAllocJobsOff = kNoAllocStatsOff + 2 * (4 * 296 + 8);
constexpr size_t kNoAllocItemsOff = kNoAllocJobsOff + 64 * (sizeof(ColJob) / sizeof(float) + 1);
constexpr size_t kNoAllocFloats = kNoAllocItemsOff + 2 * 4096;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];
constexpr int kNoAllocDevices = 64;
float* g_noalloc_ptr[kNoAllocDevices] = {nullptr};   // device address of the array, per device
std::mutex g_noalloc_mu;                              // serialises the per-device set-up

}  // namespace

extern "C" sgp_status sgp_convolve_noalloc(const float* psf, const float* f, float* out, int H, int W,
                                           int psf_origin, int transpose, void* stream) {
  if (!psf || !f || !out) return fail(SGP_ERR_ARG, "NULL array");
  sgp_shape sh{H, W, 1, 0, psf_origin};
  sgp_status st = validate_shapes(1, &sh);
  if (st) return st;
  if (size_t(H) * W > kNoAllocMaxPixels)
    return fail(SGP_ERR_SIZE_UNSUPPORTED, "sgp_convolve_noalloc supports at most 262144 pixels (e.g. 512 x 512)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the call synchronises the stream and copies from host memory, neither of which a capture allows
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    return fail(SGP_ERR_STATE, "sgp_convolve_noalloc must not be called while its stream is being captured");
  g_launch_counter = nullptr;   // no context is driven by this call
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocDevices) return fail(SGP_ERR_ARG, "device ordinal beyond the library's table (64)");
  float* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if ((st = ensure_device_ready(dev))) return st;
    if (!g_noalloc_ptr[dev]) {   // once per device: the device address of the fixed scratch array
      void* p = nullptr;
      CU(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_ptr[dev] = static_cast<float*>(p);
    }
    base = g_noalloc_ptr[dev];
  }
  const size_t P = size_t(H) * W;
  const int M = W / 2;
  float2* khat = reinterpret_cast<float2*>(base);
  float2* khatq = reinterpret_cast<float2*>(base + P);
  float* spec0 = base + P + 4 * 2048;
  float* spec1 = spec0 + P;
  double* stats = reinterpret_cast<double*>(base + kNoAllocStatsOff);
  ColJob* jobs = reinterpret_cast<ColJob*>(base + kNoAllocJobsOff);
  int2* items = reinterpret_cast<int2*>(base + kNoAllocItemsOff);
  // PSF normalisation constant
  double ps[4];
  if ((st = plane_stats(s, psf, nullptr, nullptr, P, 1, 0, stats + 8, stats))) return st;
  CU(cudaMemcpyAsync(ps, stats, sizeof(ps), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (ps[3] > 0 || !(ps[0] > 0) || !(ps[1] > 0)) return fail(SGP_ERR_PSF, "PSF must be finite with a positive sum");
  if (ps[2] < -1e-6 * ps[1]) return fail(SGP_ERR_PSF, "PSF has significantly negative samples");
  // jobs: [0] PSF spectrum, [1] convolution (or correlation); column items of both
  ColJob hj[2];
  memset(hj, 0, sizeof(hj));
  const size_t ps2 = P / 2;
  hj[0].in = reinterpret_cast<const float2*>(spec1);
  hj[0].out = khat;
  hj[0].khat = khat;
  hj[0].khatq = khatq;
  hj[0].H = H; hj[0].M = M; hj[0].nin = 1; hj[0].nout = 1; hj[0].plane_stride = ps2;
  hj[0].scale = float(1.0 / (ps[0] * double(H) * double(M)));
  hj[0].corner = psf_origin == SGP_PSF_CORNER;
  hj[1] = hj[0];
  hj[1].in = reinterpret_cast<const float2*>(spec0);
  hj[1].out = reinterpret_cast<float2*>(spec1);
  const int cpi = cols_per_item(H);
  int2 hi[2 * 1024];
  int nk = 0;
  for (int x = 0; x < M; x += cpi) hi[nk++] = make_int2(0, x);
  for (int x = 0; x < M; x += cpi) hi[nk + x / cpi] = make_int2(1, x);
  const int nc = nk;
  CU(cudaMemcpyAsync(jobs, hj, sizeof(hj), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(items, hi, sizeof(int2) * 2 * nc, cudaMemcpyHostToDevice, s));
  const int si = side_index(W), sc = side_index(H);
  const int per_view = (H + rows_per_item(W) - 1) / rows_per_item(W);
  size_t ivs = P, ovs = ps2;
  int Hh = H, one = 1, clamp = 1, noclamp = 0;
  // PSF -> spectrum plane 1 -> PSF spectrum (column pass 0)
  const float* psrc = psf;
  float2* sp1 = reinterpret_cast<float2*>(spec1);
  void* a1[] = {(void*)&psrc, (void*)&ivs, (void*)&sp1, (void*)&ovs, (void*)&Hh, (void*)&one, (void*)&clamp};
  if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view, kRowBlock, g_reg.row_smem[si], s, a1))) return st;
  const ColJob* j0 = jobs;
  const int2* it0 = items;
  int n0 = nc;
  void* a2[] = {(void*)&j0, (void*)&it0, (void*)&n0};
  if ((st = launch(g_reg.col[COL_KHAT][sc], n0, kColBlock, g_reg.col_smem[sc], s, a2))) return st;
  // f -> spectrum plane 0 -> (times PSF spectrum) plane 1 -> out
  float2* sp0 = reinterpret_cast<float2*>(spec0);
  void* a3[] = {(void*)&f, (void*)&ivs, (void*)&sp0, (void*)&ovs, (void*)&Hh, (void*)&one, (void*)&noclamp};
  if ((st = launch(g_reg.row[ROP_R2C][0][si], per_view, kRowBlock, g_reg.row_smem[si], s, a3))) return st;
  const int2* it1 = items + nc;
  void* a4[] = {(void*)&j0, (void*)&it1, (void*)&n0};
  if ((st = launch(g_reg.col[transpose ? COL_1TOP_CONJ : COL_1TOP][sc], n0, kColBlock, g_reg.col_smem[sc], s, a4)))
    return st;
  const float2* csp1 = sp1;
  float sc1 = 1.0f;
  void* a5[] = {(void*)&csp1, (void*)&ovs, (void*)&out, (void*)&ivs, (void*)&Hh, (void*)&one, (void*)&sc1};
  return launch(g_reg.row[ROP_C2R][0][si], per_view, kRowBlock, g_reg.row_smem[si], s, a5);
}
