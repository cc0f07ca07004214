// C ABI entry points: handle lifetime, argument checks, error reporting.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include <cublas_v2.h>

#include "internal.cuh"

struct stab_handle_s : StabHandle {};

static thread_local std::string g_create_err;

#define STAB_CUDA(h, call)                                                   \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return e_ == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA; \
    }                                                                        \
  } while (0)

extern "C" void stab_default_opts(stab_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gamma = 1.4;
  o->sutherland_S = 110.4 / 273.15;
  o->bulk_visc_ratio = 0.0;
  o->eps_mode = 0;
  o->eps = 0.0;
  o->gmres_m = 30;
  o->gmres_max_restarts = 200;
  o->gmres_tol = 1e-10;
  o->precond = 0;
  o->tile[0] = 8;
  o->tile[1] = 8;
  o->tile[2] = 1;
  o->precond_prec = 32;
  o->max_restarts = 300;
  o->seed = 0x5EEDULL;
  o->gmres_basis_prec = 64;
  o->stencil_prec = 64;
  o->lgmres_k = 0;
  o->precond_factor = 0;
  o->gmres_inner_m = 0;
  o->gmres_inner_tol = 1e-3;
}

static void free_handle(stab_handle h) {
  if (!h) return;
  dfree(h, h->d_q0);
  dfree(h, h->d_btab);
  dfree(h, h->d_metric);
  dfree(h, h->d_bcflags);
  dfree(h, h->d_scratch);
  dfree(h, h->d_red);
  dfree(h, h->d_gm);
  dfree(h, h->d_ir);
  dfree(h, h->d_pinv);
  dfree(h, h->d_pblk);
  dfree(h, h->d_coef);
  dfree(h, h->d_coef_f);
  dfree(h, h->d_coef_p);
  dfree(h, h->d_btab_f);
  dfree(h, h->d_btab_low);
  for (int a = 0; a < 3; ++a) {
    dfree(h, h->ax[a].tab[0]);
    dfree(h, h->ax[a].tabf[0]);
    dfree(h, h->d_dmat[a]);
    dfree(h, h->d_dmat_low[a]);
  }
  for (cudaEvent_t e : h->timer.ev) cudaEventDestroy(e);
  for (cudaGraphExec_t e : h->gm_exec)
    if (e) cudaGraphExecDestroy(e);
  if (h->cublas) cublasDestroy((cublasHandle_t)h->cublas);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

extern "C" stab_status stab_create(stab_handle* out, const double* base_flow, int base_on_device,
                                   const stab_grid* grid, double Ma, double Re, double Pr,
                                   const stab_opts* opts, void* cuda_stream) {
  if (!out) return STAB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!base_flow || !grid) { g_create_err = "stab_create: null base_flow or grid"; return STAB_ERR_INVALID_ARG; }
  const stab_grid& g = *grid;
  if (!(g.dim == 2 || g.dim == 3) || g.nx < 6 || g.ny < 6 || (g.dim == 2 && g.nz != 1) || (g.dim == 3 && g.nz < 6)) {
    g_create_err = "stab_create: need dim 2 (nz = 1) or 3, and nx, ny (nz in 3-D) >= 6";
    return STAB_ERR_INVALID_ARG;
  }
  if ((long long)g.nx * g.ny * g.nz >= (1ll << 31)) {
    g_create_err = "stab_create: at most 2^31 - 1 grid points";
    return STAB_ERR_INVALID_ARG;
  }
  if (!(g.lx > 0) || !(g.ly1 > g.ly0) || (g.dim == 3 && !(g.lz > 0)) || g.stretch < 0 || !(Ma > 0) || !(Pr > 0)) {
    g_create_err = "stab_create: invalid lengths, stretch, Mach or Prandtl number";
    return STAB_ERR_INVALID_ARG;
  }
  stab_opts o;
  if (opts) o = *opts; else stab_default_opts(&o);
  if (o.eps_mode != 0 && o.eps_mode != 2) {
    g_create_err = o.eps_mode == 1 ? "stab_create: eps_mode 1 (literal double quotient) is not implemented on the GPU"
                                   : "stab_create: eps_mode must be 0 or 2";
    return o.eps_mode == 1 ? STAB_ERR_UNSUPPORTED : STAB_ERR_INVALID_ARG;
  }
  if (o.gmres_m < 1 || o.gmres_m > 200 || !(o.gmres_tol > 0) || o.gmres_max_restarts < 1 || o.eps < 0 ||
      !(o.gamma > 1) || o.sutherland_S < 0 || o.bulk_visc_ratio < 0 || o.max_restarts < 0 ||
      (o.precond_prec != 16 && o.precond_prec != 32 && o.precond_prec != 64) || (o.precond < 0 || o.precond > 2) ||
      (o.gmres_basis_prec != 32 && o.gmres_basis_prec != 64) || (o.stencil_prec != 48 && o.stencil_prec != 64)) {
    g_create_err = "stab_create: invalid option value";
    return STAB_ERR_INVALID_ARG;
  }
  if (o.gmres_inner_m < 0 || o.gmres_inner_m > 100 || !(o.gmres_inner_tol >= 0.0 && o.gmres_inner_tol < 1.0)) {
    g_create_err = "stab_create: gmres_inner_m must be in [0, 100] and gmres_inner_tol in [0, 1)";
    return STAB_ERR_INVALID_ARG;
  }
  if (o.gmres_inner_m > 0 && (o.gmres_basis_prec != 64 || o.lgmres_k > 0)) {
    g_create_err = "stab_create: the nested inner solver needs the FP64 outer basis and no LGMRES";
    return STAB_ERR_UNSUPPORTED;
  }
  if (o.precond == 2 && o.precond_prec == 16) {
    g_create_err = "stab_create: the reduced-operator preconditioner (precond 2) stores FP32 or FP64 factors";
    return STAB_ERR_UNSUPPORTED;
  }
  if (o.precond_factor < 0 || o.precond_factor > 2) {
    g_create_err = "stab_create: precond_factor must be 0, 1 or 2";
    return STAB_ERR_INVALID_ARG;
  }
  if (o.lgmres_k < 0 || o.lgmres_k > STAB_MAX_LGMRES_K || (o.lgmres_k > 0 && o.lgmres_k >= o.gmres_m)) {
    g_create_err = "stab_create: lgmres_k must be in [0, min(8, gmres_m - 1)]";
    return STAB_ERR_INVALID_ARG;
  }
  if (o.lgmres_k > 0 && o.gmres_basis_prec != 64) {
    g_create_err = "stab_create: LGMRES (lgmres_k > 0) needs the FP64 GMRES basis";
    return STAB_ERR_UNSUPPORTED;
  }
  stab_handle h = new (std::nothrow) stab_handle_s();
  if (!h) return STAB_ERR_OOM;
  h->dim = g.dim; h->nx = g.nx; h->ny = g.ny; h->nz = g.nz; h->nv = g.dim + 2;
  h->npts = (long long)g.nx * g.ny * g.nz;
  h->n = h->nv * h->npts;
  h->lx = g.lx; h->ly0 = g.ly0; h->ly1 = g.ly1; h->lz = g.lz; h->stretch = g.stretch;
  h->gamma = o.gamma; h->Ma = Ma; h->Re = Re; h->Pr = Pr; h->S = o.sutherland_S; h->bulk = o.bulk_visc_ratio;
  h->R = 1.0 / (o.gamma * Ma * Ma);
  h->cp = o.gamma * h->R / (o.gamma - 1.0);
  h->visc = Re > 0.0;
  h->opts = o;
  h->stencil_ff = o.stencil_prec == 48 ? 1 : 0;
  h->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&h->device);
  h->last_eps_mode = -1;
  // host copy of the base state: homogeneity test, norm, boundary flags
  std::vector<double> q0((size_t)h->n);
  cudaError_t e;
  if (base_on_device) {
    e = cudaMemcpyAsync(q0.data(), base_flow, h->n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  else { std::memcpy(q0.data(), base_flow, h->n * sizeof(double)); e = cudaSuccess; }
  if (e != cudaSuccess) { g_create_err = std::string("stab_create: copy of base_flow: ") + cudaGetErrorString(e); free_handle(h); return STAB_ERR_CUDA; }
  double nrm = 0.0;
  bool finite = true, homog = true;
  for (long long a = 0; a < h->n; ++a) { nrm += q0[a] * q0[a]; if (!std::isfinite(q0[a])) finite = false; }
  for (int var = 0; var < h->nv && homog; ++var)
    for (int k = 0; k < h->nz && homog; ++k)
      for (int j = 0; j < h->ny && homog; ++j) {
        const double* row = q0.data() + (long long)var * h->npts + ((long long)k * h->ny + j) * h->nx;
        const double* ref = q0.data() + (long long)var * h->npts + (long long)j * h->nx;
        for (int i = 0; i < h->nx; ++i) if (row[i] != ref[0]) { homog = false; break; }
      }
  bool positive = true;
  for (long long a = 0; a < h->npts; ++a) if (!(q0[a] > 0)) positive = false;
  if (!finite || !positive) { g_create_err = "stab_create: base_flow must be finite with positive pressure"; free_handle(h); return STAB_ERR_INVALID_ARG; }
  h->q0norm = std::sqrt(nrm);
  h->homog = homog;
  h->nbase = homog ? h->ny : h->npts;
  e = dalloc(h, &h->d_q0, h->n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_q0, q0.data(), h->n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = jv_setup(h, q0.data());
  if (e == cudaSuccess) e = kry_init_attributes();
  if (e != cudaSuccess) {
    g_create_err = std::string("stab_create: ") + cudaGetErrorString(e);
    stab_status st = e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA;
    free_handle(h);
    return st;
  }
  jv_tune_apply_cached(h);
  *out = h;
  return STAB_OK;
}

extern "C" void stab_destroy(stab_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

extern "C" const char* stab_last_error(stab_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

// message for entry points that take no handle (reported by stab_last_error(NULL))
void stab_set_global_error(const char* msg) { g_create_err = msg ? msg : ""; }

extern "C" long long stab_size(stab_handle h) { return h ? h->n : 0; }

extern "C" stab_status stab_apply_J(stab_handle h, const void* v, void* Jv, double shift_re, double shift_im) {
  if (!h) return STAB_ERR_INVALID_ARG;
  if (!v || !Jv) { h->err = "stab_apply_J: null vector"; return STAB_ERR_INVALID_ARG; }
  const char* a = (const char*)v;
  const char* b = (const char*)Jv;
  const long long bytes = h->n * (long long)sizeof(double2);
  if (a < b + bytes && b < a + bytes) { h->err = "stab_apply_J: v and Jv overlap"; return STAB_ERR_INVALID_ARG; }
  STAB_CUDA(h, jv_apply(h, (const double2*)v, (double2*)Jv, make_double2(shift_re, shift_im), h->opts.eps_mode));
  return STAB_OK;
}

extern "C" stab_status stab_last_eps(stab_handle h, double* eps) {
  if (!h || !eps) return STAB_ERR_INVALID_ARG;
  STAB_CUDA(h, cudaMemcpyAsync(eps, h->d_eps, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  STAB_CUDA(h, cudaStreamSynchronize(h->stream));
  return STAB_OK;
}

// ---------------------------------------------------------------------------
// Device memory: one library-owned, stream-ordered pool per device.  Handles
// allocate and free on their own stream (no device-wide synchronisation, so
// handles on different streams run side by side); freed memory stays cached
// in the pool for later handles until stab_trim_memory.
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaError_t dev_alloc(StabHandle* h, void** p, size_t bytes) { return dev_alloc_stream(h->device, h->stream, p, bytes); }

cudaError_t dev_alloc_stream(int dev, cudaStream_t stream, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
      if (e != cudaSuccess) { g_pool[dev] = nullptr; return e; }
      unsigned long long keep = ~0ULL;
      cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

void dev_free(StabHandle* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

extern "C" int stab_trim_memory(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  int count = 0;
  for (int d = 0; d < 64; ++d)
    if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) == cudaSuccess) ++count;
  return count;
}

// ---------------------------------------------------------------------------
// phase timing
int phase_begin(StabHandle* h, int phase) {
  PhaseTimer& T = h->timer;
  if (!T.on || h->capturing) return -1;
  if (T.used >= PhaseTimer::kMax) { ++T.dropped; return -1; }
  const int slot = T.used;
  while ((int)T.ev.size() < 2 * (slot + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { ++T.dropped; return -1; }
    T.ev.push_back(e);
  }
  if ((int)T.phase.size() <= slot) T.phase.resize(slot + 1);
  T.phase[slot] = phase;
  if (cudaEventRecord(T.ev[2 * slot], h->stream) != cudaSuccess) { ++T.dropped; return -1; }
  T.used = slot + 1;
  return slot;
}

void phase_end(StabHandle* h, int slot) {
  if (slot < 0) return;
  cudaEventRecord(h->timer.ev[2 * slot + 1], h->stream);
}

extern "C" stab_status stab_timing(stab_handle h, int enable) {
  if (!h) return STAB_ERR_INVALID_ARG;
  STAB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->timer.on = enable != 0;
  h->timer.used = 0;
  h->timer.dropped = 0;
  return STAB_OK;
}

extern "C" stab_status stab_timing_read(stab_handle h, double* ms, long long* count, long long* dropped) {
  if (!h) return STAB_ERR_INVALID_ARG;
  STAB_CUDA(h, cudaStreamSynchronize(h->stream));
  double acc[STAB_PHASE_COUNT] = {0};
  long long cnt[STAB_PHASE_COUNT] = {0};
  PhaseTimer& T = h->timer;
  for (int i = 0; i < T.used; ++i) {
    float t = 0.f;
    STAB_CUDA(h, cudaEventElapsedTime(&t, T.ev[2 * i], T.ev[2 * i + 1]));
    const int p = T.phase[i];
    if (p >= 0 && p < STAB_PHASE_COUNT) { acc[p] += t; cnt[p]++; }
  }
  if (ms) for (int p = 0; p < STAB_PHASE_COUNT; ++p) ms[p] = acc[p];
  if (count) for (int p = 0; p < STAB_PHASE_COUNT; ++p) count[p] = cnt[p];
  if (dropped) *dropped = T.dropped;
  T.used = 0;
  T.dropped = 0;
  return STAB_OK;
}

extern "C" stab_status stab_autotune(stab_handle h, int force, int* cfg, double* ms) {
  if (!h) return STAB_ERR_INVALID_ARG;
  double t[3] = {0.0, 0.0, 0.0};
  STAB_CUDA(h, jv_autotune(h, force, t));
  if (cfg)
    for (int a = 0; a < 3; ++a) {
      cfg[3 * a] = a < h->dim ? h->line_cfg[a].C : 0;
      cfg[3 * a + 1] = a < h->dim ? h->line_cfg[a].L : 0;
      cfg[3 * a + 2] = a < h->dim ? h->line_cfg[a].kp : 0;
    }
  if (ms)
    for (int a = 0; a < 3; ++a) ms[a] = a < h->dim ? t[a] : 0.0;
  return STAB_OK;
}

extern "C" stab_status stab_set_line_config(stab_handle h, int axis, int C, int L, int kinds) {
  if (!h) return STAB_ERR_INVALID_ARG;
  if (axis < 0 || axis >= h->dim) { h->err = "stab_set_line_config: bad axis"; return STAB_ERR_INVALID_ARG; }
  if (C == 0 && L == 0 && kinds == 0) { h->line_cfg[axis] = LineCfg{}; return STAB_OK; }
  const int n = h->ax[axis].n;
  const long long LS = n + (n >> 5) + 1;
  const int nch = (C > 0) ? (n + C - 1) / C : 0;
  const int tpl = (kinds == 2 ? 4 : 2) * nch, planes = kinds == 3 ? 2 : 2 + 2 * kinds;
  if ((C != 16 && C != 32 && C != 64) || L < 1 || L > 32 || kinds < 1 || kinds > 3 ||
      tpl * L > (kinds == 3 ? 512 : 1024) || planes * 8 * LS * L + 16 > 200 * 1024) {
    h->err = "stab_set_line_config: C must be 16, 32 or 64, L in 1..32 and kinds 1, 2 or 3, within 1024 threads "
             "(512 with kinds 3) and 200 KB";
    return STAB_ERR_INVALID_ARG;
  }
  h->line_cfg[axis] = LineCfg{C, L, kinds};
  return STAB_OK;
}

extern "C" int stab_autotune_save(const char* path) { return path ? jv_tune_save(path) : -1; }
extern "C" int stab_autotune_load(const char* path) { return path ? jv_tune_load(path) : -1; }

extern "C" stab_status stab_get_stats(stab_handle h, stab_stats* s) {
  if (!h || !s) return STAB_ERR_INVALID_ARG;
  *s = h->stats;
  return STAB_OK;
}
