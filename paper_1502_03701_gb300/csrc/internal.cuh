// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/stab.h"

#define STAB_MAX_DIM 3
#define STAB_MAX_JOBS 16
#define STAB_MAX_LGMRES_K 8

// ---------------------------------------------------------------------------
// Compact-scheme line solve tables for one axis (device pointers).
// Kind 0 = first derivative, kind 1 = second derivative.  The implicit
// tridiagonal system is solved as a forward sweep g_t = r_t - l_t g_{t-1}
// followed by a backward sweep x_t = g_t dinv_t - m_t x_{t+1}: Thomas
// elimination for bounded lines, the two first-order factors of the
// circulant matrix for periodic lines.
// ---------------------------------------------------------------------------
struct AxisTables {
  int n;
  int periodic;
  double h;
  int K[2];             // warm-up length of a chunked sweep (influence decays below 2^-56)
  int Wn[2];            // near part of the warm-up kept in FP64 (the rest runs in FP32)
  double pdinv[2];      // periodic: 1/c of the factorised circulant, per kind (folded into the stencil)
  float* tabf[2];       // device FP32 copies [l'(n), m(n)] per kind (far warm-up)
  double* tab[2];       // device, per kind: [l'(n), dinv(n), m(n)]: Thomas factors of the sweep on the
                        // right-hand side scaled by dinv (l'_t = l_t d_{t-1} / d_t)
};

struct LineJob {
  const double2* in;
  double2* out1;  // first derivative (nullable)
  double2* out2;  // second derivative (nullable)
};

// Scratch / base-table slot layout for a problem of dimension D.
// Field f: 0 = p, 1..D = u_i, D+1 = s, D+2 = T.   Second-derivative field g:
// 0..D-1 = u_i, D = T.   mix[i][k] = d/dx_i d/dx_k u_k (i != k).
struct Slots {
  int Tw;
  int d1[3][6];
  int d2[3][4];
  int mix[3][3];
  int count;
};

// What a captured GMRES cycle graph depends on (replayed while unchanged).
struct GmGraphKey {
  bool valid = false;
  double sigma_re = 0, sigma_im = 0;
  int eps_mode = -1, m = 0, pc = 0, pprec = 0, basis = 64, lgk = 0, naug = 0, mi = 0;
  const void* ws = nullptr;
  const void* pinv = nullptr;
  long long n = 0;
  bool operator==(const GmGraphKey& o) const {
    return valid && o.valid && sigma_re == o.sigma_re && sigma_im == o.sigma_im && eps_mode == o.eps_mode &&
           m == o.m && pc == o.pc && pprec == o.pprec && ws == o.ws && pinv == o.pinv && n == o.n &&
           basis == o.basis && lgk == o.lgk && naug == o.naug && mi == o.mi;
  }
};

// Launch shape of the compact-derivative line pass along one axis: C points
// per sweep chunk, L lines per CTA, kp derivative kinds at once (0: built-in
// default).
struct LineCfg {
  int C = 0, L = 0, kp = 0;
};

// Event pairs around library phases (stab_timing); recording is a no-op
// unless enabled.
struct PhaseTimer {
  static constexpr int kMax = 65536;
  bool on = false;
  std::vector<cudaEvent_t> ev;       // pool, reused after every read
  std::vector<int> phase;            // per interval
  int used = 0;                      // intervals recorded since the last read
  long long dropped = 0;
};

struct StabHandle {
  // problem
  int dim, nx, ny, nz, nv;
  long long npts, n;
  double lx, ly0, ly1, lz, stretch;
  double gamma, Ma, Re, Pr, S, bulk;
  double R, cp;
  bool visc;
  bool homog;        // base state depends on y only
  long long nbase;   // ny if homog else npts
  double q0norm;
  stab_opts opts;
  cudaStream_t stream;
  int device = 0;  // current device at stab_create; the handle's memory lives there
  Slots slots;
  AxisTables ax[3];
  // device memory
  double* d_q0;          // base state, n doubles
  double* d_btab;        // base tables (see jv.cu)
  double* d_metric;      // eta_y[ny], eta_yy[ny]
  unsigned char* d_bcflags;  // [2][nz*nx]
  double2* d_scratch;    // slots.count * npts complex
  double* d_red;         // reduction partials (red_blocks) + scalars
  int red_blocks;
  double* d_eps;         // scalar: epsilon of the last J v
  int last_eps_mode;
  int stencil_ff;        // 1: compact-scheme right-hand sides of J v in FP32 pairs (stencil_prec 48)
  // Krylov workspace (allocated on demand, grown as needed)
  double2* d_gm;   // GMRES
  size_t gm_elems;
  double2* d_ir;   // IRAM
  size_t ir_elems;
  // block-Jacobi preconditioner
  void* d_pinv;          // inverses, FP64 or FP32 complex
  double2* d_pblk;       // assembled blocks (FP64) scratch for the build
  long long ntiles, bsize;
  double psigma_re, psigma_im;
  bool pvalid;
  int pprec;
  double* d_dmat[3];     // dense 1-D derivative matrices [kind][n*n] per axis (assembly)
  double* d_dmat_low[3] = {nullptr, nullptr, nullptr};  // the reduced operator's (second-order explicit)
  double* d_btab_low = nullptr;  // base tables with the reduced operator's derivatives
  double* d_coef;        // per-row tangent coefficients of the pointwise map (y-only base)
  double* d_coef_f;      // the same with the y metric folded in (inputs: eta-derivatives)
  struct ffn* d_coef_p;  // d_coef_f as FP32 pairs (hi, lo), read by the pointwise kernel
  float* d_btab_f;       // FP32 copy of the base tables (for the O(eps) remainder)
  bool force_dn_path;    // use the full FP64 difference-number pointwise kernel
  void* cublas = nullptr;  // cuBLAS handle of the tensor-core block factorisation (created on first use)
  // statistics
  stab_stats stats;
  PhaseTimer timer;
  LineCfg line_cfg[3];  // per axis, from stab_autotune
  // graph capture of the GMRES cycle (solver.cu): while gate is set, the
  // gated kernels launched by jv_apply, pc_apply, kry_cgs2 and kry_scale
  // return at once when *gate != 0 (the cycle has converged)
  const int* gate = nullptr;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gm_exec[STAB_MAX_LGMRES_K + 1] = {};  // per number of augmentation vectors (LGMRES)
  GmGraphKey gm_key[STAB_MAX_LGMRES_K + 1];
  std::string err;
};

// api.cu: stream-ordered device memory from the library's pool on the
// handle's stream (dalloc: typed wrapper).
cudaError_t dev_alloc(StabHandle* h, void** p, size_t bytes);
cudaError_t dev_alloc_stream(int device, cudaStream_t stream, void** p, size_t bytes);
void dev_free(StabHandle* h, void* p);
template <class T>
inline cudaError_t dalloc(StabHandle* h, T** p, size_t bytes) {
  return dev_alloc(h, (void**)p, bytes);
}
inline void dfree(StabHandle* h, const void* p) { dev_free(h, const_cast<void*>(p)); }

// api.cu: phase timing.  phase_begin returns the interval's slot (or -1 when
// not recording); phase_end records its closing event.
int phase_begin(StabHandle* h, int phase);
void phase_end(StabHandle* h, int slot);

// jv.cu
cudaError_t jv_setup(StabHandle* h, const double* q0_host);
cudaError_t jv_apply(StabHandle* h, const double2* v, double2* out, double2 shift, int eps_mode);
cudaError_t launch_norm2(StabHandle* h, const double2* v, long long n, double* d_out, int mode);
cudaError_t jv_autotune(StabHandle* h, int force, double* ms_out);
int jv_tune_save(const char* path);
int jv_tune_load(const char* path);
void jv_tune_apply_cached(StabHandle* h);
cudaError_t jv_derivative_matrices(StabHandle* h, int axis, double2* work, double2* out1, double2* out2);
// base tables of the reduced operator (second-order explicit derivatives of the base fields) into btab
cudaError_t jv_reduced_base_table(StabHandle* h, double* btab);

// krylov.cu
cudaError_t kry_dot(StabHandle* h, const double2* V, int k, long long n, const double2* w, double2* d_h,
                    double2* partial, int accumulate);
cudaError_t kry_gemv_sub(StabHandle* h, const double2* V, int k, long long n, const double2* d_h, double2* w);
cudaError_t kry_gemv_add(StabHandle* h, const double2* V, int k, long long n, const double2* d_y, double2* x,
                         const int* kdev = nullptr);
cudaError_t kry_cgs2(StabHandle* h, const double2* V, int k, long long n, double2* w, double2* d_h2k, double* d_norm,
                     double2* partial);
cudaError_t kry_scale(StabHandle* h, double2* x, long long n, const double* d_norm, double2* out_or_null);
cudaError_t kry_axpby(StabHandle* h, double2 a, const double2* x, double2 b, double2* y, long long n);
cudaError_t kry_copy(StabHandle* h, const double2* x, double2* y, long long n);
cudaError_t kry_update_basis(StabHandle* h, double2* V, int m, int kk, long long n, const double2* d_Q, double2* tmp);
int kry_partial_elems(long long n, int k);
int kry_dgks_partial_elems(long long n, int k);
cudaError_t kry_dgks(StabHandle* h, const double2* V, int k, long long n, double2* w, double2* d_h, double* d_norm,
                     double2* partial);
cudaError_t kry_dgks32(StabHandle* h, const float2* V, int k, long long n, float2* w, double2* d_h, double* d_norm,
                       double2* partial);
cudaError_t kry_to_f32(StabHandle* h, const double2* in, long long n, const double* d_norm, float2* out);
cudaError_t kry_scale32(StabHandle* h, float2* x, long long n, const double* d_norm);
cudaError_t kry_to_f64(StabHandle* h, const float2* in, long long n, double2* out);
cudaError_t kry_gemv32(StabHandle* h, const float2* V, int k, const int* kdev, long long n, const double2* y,
                       double2* out);
cudaError_t kry_init_attributes();
cudaError_t kry_cgs2_stream(cudaStream_t st, const double2* V, int k, long long n, double2* w, double2* d_h,
                            double* d_norm, double2* partial, double* norm_partial, int norm_blocks);
cudaError_t launch_norm2_stream(cudaStream_t st, const double2* v, long long n, double* partial, int nb,
                                double* d_out);

// precond.cu
cudaError_t pc_build(StabHandle* h, double2 sigma);
cudaError_t pc_apply(StabHandle* h, const double2* q, double2* z, const float2* q32 = nullptr);
cudaError_t pc_block(StabHandle* h, double2 sigma, long long t, double2* d_out);


// ---------------------------------------------------------------------------
// Batches of handles (stab_jv_batch_*): per-call parameter images of the
// batched kernels.  An image holds, per launch, the instances' items followed
// by the block offsets start[0..count] (item i owns blocks [start[i],
// start[i+1])), each section 16-byte aligned; batch_stage copies it to the
// batch's device buffer through a pinned staging buffer.
// ---------------------------------------------------------------------------
struct stab_jv_batch_s {
  std::vector<StabHandle*> hs;
  int device = 0;
  cudaStream_t stream = nullptr;
  void* d_buf = nullptr;
  size_t d_cap = 0;
  void* h_buf = nullptr;  // pinned
  size_t h_cap = 0;
  cudaEvent_t copied = nullptr;  // the last transfer out of h_buf has completed
  cudaEvent_t order = nullptr;   // orders the batch's stream against its handles' streams
  std::string err;
};

struct BatchSection {
  size_t items = 0, start = 0;  // byte offsets in the image
  int count = 0, blocks = 0, threads = 0;
  size_t smem = 0;
};

struct BatchImage {
  std::vector<unsigned char> bytes;
  bool overflow = false;  // a section's block count does not fit a launch (batch_stage refuses the image)
  size_t put(const void* p, size_t n) {
    const size_t off = (bytes.size() + 15) & ~(size_t)15;
    bytes.resize(off + n);
    if (n) std::memcpy(bytes.data() + off, p, n);
    return off;
  }
  template <class T>
  BatchSection section(const std::vector<T>& items, const std::vector<int>& blocks, int threads, size_t smem) {
    BatchSection s;
    s.count = (int)items.size();
    if (!s.count) return s;
    std::vector<int> start(items.size() + 1, 0);
    long long total = 0;
    for (size_t i = 0; i < items.size(); ++i) {
      total += blocks[i];
      if (blocks[i] < 0 || total > 0x7FFFFFFFLL) {  // grid x and the int offsets are limited to 2^31 - 1
        overflow = true;
        total = 0;
      }
      start[i + 1] = (int)total;
    }
    s.items = put(items.data(), items.size() * sizeof(T));
    s.start = put(start.data(), start.size() * sizeof(int));
    s.blocks = start.back();
    s.threads = threads;
    s.smem = smem;
    return s;
  }
};

cudaError_t batch_stage(stab_jv_batch_s* B, const BatchImage& im);

// Planned batched phases: the sections of a parameter image (built once,
// copied to the device once) and the launches that read them.  gates[i]
// (nullable) skips instance i's work while *gates[i] != 0.
struct JvBatchPlan {
  BatchSection norm, temp, line[3][4], point[2];
  std::vector<double*> zero_eps;  // epsilon slots of the exact-tangent instances
};
cudaError_t jv_batch_plan(const std::vector<StabHandle*>& hs, const double2* const* v, double2* const* out,
                          const double2* shifts, const int* const* gates, BatchImage& im, JvBatchPlan& plan);
cudaError_t jv_batch_launch(const JvBatchPlan& plan, const unsigned char* d, cudaStream_t st);
cudaError_t jv_batch_zero_eps(const JvBatchPlan& plan, cudaStream_t st);
struct NormJob {  // ||v|| into *out with the reduction scratch of handle h
  StabHandle* h;
  const double2* v;
  long long n;
  double* out;
  int mode;  // 0: sum of squares, 1: norm
  const int* gate;
};
cudaError_t norm_batch_plan(const std::vector<NormJob>& jobs, BatchImage& im, BatchSection& sec);
cudaError_t norm_batch_launch(const BatchSection& sec, const unsigned char* d, cudaStream_t st);
struct PcBatchPlan {
  BatchSection sec[4];
};
cudaError_t pc_batch_plan(const std::vector<StabHandle*>& hs, const double2* const* q, double2* const* z,
                          const int* const* gates, BatchImage& im, PcBatchPlan& plan);
cudaError_t pc_batch_launch(const PcBatchPlan& plan, const unsigned char* d, cudaStream_t st);
struct CgsBatchPlan {
  BatchSection S, N;
  size_t sm = 0;
};
// Order the batch's stream after the work queued so far on every handle's own
// stream (begin), and every handle's stream after the batch's launches (end),
// so that a batch call and single-handle calls on other streams never race on
// a handle's scratch.
cudaError_t batch_order_begin(stab_jv_batch_s* B);
cudaError_t batch_order_end(stab_jv_batch_s* B);
struct CgsJob {  // one instance of a batched CGS2 (scratch as for kry_cgs2)
  const double2* V;
  int k;
  long long n;
  double2* w;
  double2* d_h;
  double* d_norm;
  double2* partial;
  const int* gate = nullptr;
};
cudaError_t kry_cgs2_batch(stab_jv_batch_s* B, const std::vector<CgsJob>& jobs);
cudaError_t cgs2_batch_plan(const std::vector<CgsJob>& jobs, BatchImage& im, CgsBatchPlan& plan);
cudaError_t cgs2_batch_launch(const CgsBatchPlan& plan, const unsigned char* d, cudaStream_t st);
cudaError_t pc_apply_batch(stab_jv_batch_s* B, const double2* const* q, double2* const* z);
