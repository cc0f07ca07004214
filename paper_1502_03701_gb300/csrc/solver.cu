// Inner linear solver and outer eigensolver, orchestrated from the host with
// all vector work on the device:
//  * restarted GMRES(m) (Sec. "Iterative solvers") in flexible,
//    right-preconditioned form, x0 = 0, stopping on ||b - A x|| <= tol ||b||;
//  * the Cayley-transformed implicitly restarted Arnoldi method
//    (Algorithm iram, Eqs. cayley_transform / cayley_arnoldi / ritz_estimate)
//    with CGS2 orthogonalisation and exact shifts.
// The small (m x m) Hessenberg algebra of the restart stays on the device
// (k_restart), and so does GMRES's Givens least-squares update (k_gm_step):
// a GMRES cycle is one replayed CUDA graph and one host read.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "hess_dev.cuh"
#include "internal.cuh"

typedef std::complex<double> cd;

namespace {

struct Fail {
  stab_status st;
};

inline void ck(StabHandle* h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
    throw Fail{e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA};
  }
}

inline void fail(StabHandle* h, stab_status st, const std::string& msg) {
  h->err = msg;
  throw Fail{st};
}

inline double2 d2(cd z) { return make_double2(z.real(), z.imag()); }

// grow-only device workspace
double2* ensure(StabHandle* h, double2** p, size_t* have, size_t need) {
  if (*have >= need) return *p;
  dfree(h, *p);
  *p = nullptr;
  *have = 0;
  ck(h, dalloc(h, p, need * sizeof(double2)), "workspace allocation");
  *have = need;
  return *p;
}

// GMRES workspace layout (complex elements).  FP64 basis: V, Z (flexible).
// FP32 basis: V32, and FP64 work vectors w (J z), zt (preconditioned
// direction or correction) and t (V32 y).
struct GmresWs {
  double2 *V, *Z, *r, *b, *x, *partial, *dh, *y;
  double* dnorm;
  float2* V32;
  double2 *w, *zt, *t;
};

constexpr int kMaxGmresM = 200;  // stab_create rejects larger gmres_m
constexpr long long kSelectiveMinN = 16384;  // unknowns from which GMRES uses selective reorthogonalisation

// Device-resident least-squares state of one GMRES cycle: the rotated
// Hessenberg columns R (m x m, row-major), the rotated right-hand side g,
// the Givens rotations (cs, sn), flags [done, jend, status] and the scalars
// [tol ||b||, |g_{j+1}|].
struct GmDev {
  hd::zc *R, *g, *sn;
  double* cs;
  int* flags;
  double* sc;
  const double2* dh;
  const double* dnorm;
  double2* y;
  int m;
};

struct GmReport {  // read by the host once per cycle
  double beta;     // ||b - A x|| after the cycle
  int jend;        // iterations performed in the cycle
  int status;      // 0, or 1 when a Krylov quantity was not finite
};

GmresWs gmres_ws(StabHandle* h, GmDev* D, GmReport** rep) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond == 1;
  const bool b32 = h->opts.gmres_basis_prec == 32;
  const size_t part = (size_t)std::max(kry_partial_elems(n, m + 1), kry_dgks_partial_elems(n, m + 1));
  const size_t small = (size_t)m * m + (m + 1) + m + (m + 1) / 2 + 1 + 4 + 4;
  const size_t basis = b32 ? ((size_t)(m + 1) * n + 1) / 2 : (size_t)(m + 1) * n + (pc ? (size_t)m * n : 0);
  const size_t work = b32 ? 6 * (size_t)n : 3 * (size_t)n;
  size_t need = basis + work + part + 2 * (m + 1) + (m + 1) + 4 + small;
  double2* base = ensure(h, &h->d_gm, &h->gm_elems, need);
  GmresWs w{};
  if (b32) {
    w.V32 = (float2*)base;
  } else {
    w.V = base;
    w.Z = pc ? base + (size_t)(m + 1) * n : nullptr;
  }
  w.r = base + basis;
  w.b = w.r + n;
  w.x = w.b + n;
  double2* q = w.x + n;
  if (b32) {
    w.w = q;
    w.zt = q + n;
    w.t = q + 2 * n;
    q += 3 * n;
  }
  w.partial = q;
  w.dh = w.partial + part;
  w.y = w.dh + 2 * (m + 1);
  w.dnorm = (double*)(w.y + (m + 1));
  double2* p = w.y + (m + 1) + 4;
  D->R = (hd::zc*)p; p += (size_t)m * m;
  D->g = (hd::zc*)p; p += m + 1;
  D->sn = (hd::zc*)p; p += m;
  D->cs = (double*)p; p += (m + 1) / 2 + 1;
  D->flags = (int*)p; p += 1;        // 4 ints
  D->sc = (double*)p; p += 1;        // 2 doubles
  *rep = (GmReport*)p; p += 1;       // 16 bytes
  D->dh = w.dh;
  D->dnorm = w.dnorm;
  D->y = w.y;
  D->m = m;
  return w;
}

double read_scalar(StabHandle* h, const double* d) {
  double v;
  ck(h, cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read scalar");
  ck(h, cudaStreamSynchronize(h->stream), "sync");
  return v;
}

__global__ void k_gm_tol(GmDev d, double tol) { d.sc[0] = tol * (*d.dnorm); }

// start of a cycle: g = (beta, 0, ...), beta = ||r|| (in dnorm)
__global__ void k_gm_cycle_init(GmDev d) {
  if (threadIdx.x == 0) {
    d.flags[0] = 0;
    d.flags[1] = 0;
    d.flags[2] = 0;
  }
  for (int i = threadIdx.x; i <= d.m; i += blockDim.x) d.g[i] = hd::mk(i == 0 ? *d.dnorm : 0.0);
}

__device__ __forceinline__ bool finite_zc(hd::zc z) { return fabs(z.re) < INFINITY && fabs(z.im) < INFINITY; }

// Arnoldi column j (h_0..h_j from CGS2, h_{j+1} = ||w||): previous rotations,
// the new rotation that annihilates h_{j+1}, the rotated right-hand side and
// the convergence test |g_{j+1}| <= tol ||b|| (or w = 0).  One warp: the
// column and the rotations are staged in shared memory by all lanes, the
// rotation chain runs on lane 0.
__global__ void k_gm_step(GmDev d, int j) {
  __shared__ hd::zc col[kMaxGmresM + 1], sn[kMaxGmresM];
  __shared__ double cs[kMaxGmresM];
  if (d.flags[0]) return;
  const int m = d.m, lane = threadIdx.x;
  const double wn = *d.dnorm;
  int bad = !(fabs(wn) < INFINITY);
  for (int i = lane; i <= j; i += 32) {
    const hd::zc v = hd::mk(d.dh[i].x, d.dh[i].y);
    bad |= !finite_zc(v);
    col[i] = v;
  }
  for (int i = lane; i < j; i += 32) {
    cs[i] = d.cs[i];
    sn[i] = d.sn[i];
  }
  bad = __any_sync(0xffffffffu, bad);
  __syncwarp();
  if (bad) {
    if (lane == 0) { d.flags[2] = 1; d.flags[0] = 1; }
    return;
  }
  if (lane == 0) {
    for (int i = 0; i < j; ++i) {
      const hd::zc a = col[i], b = col[i + 1];
      col[i] = cs[i] * a + sn[i] * b;
      col[i + 1] = cs[i] * b - hd::conj(sn[i]) * a;
    }
    double c;
    hd::zc s;
    const hd::zc sub = hd::mk(wn);
    hd::givens(col[j], sub, c, s);
    d.cs[j] = c;
    d.sn[j] = s;
    col[j] = c * col[j] + s * sub;
    const hd::zc gj = d.g[j];
    d.g[j + 1] = -(hd::conj(s) * gj);
    d.g[j] = c * gj;
    d.flags[1] = j + 1;
    const double res = hd::zabs(d.g[j + 1]);
    d.sc[1] = res;
    if (res <= d.sc[0] || wn == 0.0) d.flags[0] = 1;
  }
  __syncwarp();
  for (int i = lane; i <= j; i += 32) d.R[i * m + j] = col[i];
}

// y = R^{-1} g over the jend columns of the cycle, by columns: y_i from the
// diagonal, then every thread removes y_i's contribution from its rows.
__global__ void k_gm_solve(GmDev d) {
  __shared__ hd::zc s[kMaxGmresM];
  __shared__ hd::zc yi;
  const int m = d.m, je = d.flags[1];
  for (int l = threadIdx.x; l < je; l += blockDim.x) s[l] = d.g[l];
  __syncthreads();
  for (int i = je - 1; i >= 0; --i) {
    if (threadIdx.x == 0) {
      yi = s[i] / d.R[i * m + i];
      d.y[i] = make_double2(yi.re, yi.im);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < i; l += blockDim.x) s[l] = s[l] - d.R[l * m + i] * yi;
    __syncthreads();
  }
}

__global__ void k_gm_report(GmDev d, GmReport* rep) {
  rep->beta = *d.dnorm;
  rep->jend = d.flags[1];
  rep->status = d.flags[2];
}

// One GMRES cycle as a CUDA graph: V_0 = r / beta; m Arnoldi steps, each
// (right preconditioner, J v - sigma v, Gram-Schmidt with selective
// reorthogonalisation, Givens update, scaling) gated
// on the device flag that the Givens update raises at convergence; the
// least-squares solve, x += Z y (V y), and the true residual r = b - A x with
// its norm.  Captured once per handle, shift and workspace, replayed for
// every cycle of every solve: the host only reads the report once per cycle.
cudaGraphExec_t gm_graph(StabHandle* h, cd sigma, int eps_mode, const GmresWs& W, const GmDev& D, GmReport* rep) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond == 1;
  GmGraphKey key;
  key.valid = true;
  key.sigma_re = sigma.real();
  key.sigma_im = sigma.imag();
  key.eps_mode = eps_mode;
  key.m = m;
  key.pc = pc;
  key.pprec = h->pprec;
  key.ws = h->d_gm;
  key.pinv = pc ? h->d_pinv : nullptr;
  key.n = n;
  key.basis = h->opts.gmres_basis_prec;
  if (h->gm_exec && key == h->gm_key) return h->gm_exec;
  if (h->gm_exec) {
    cudaGraphExecDestroy(h->gm_exec);
    h->gm_exec = nullptr;
    h->gm_key.valid = false;
  }
  if (!h->cap_stream) ck(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
  const stab_stats saved_stats = h->stats;
  cudaStream_t saved_stream = h->stream;
  h->stream = h->cap_stream;
  h->capturing = true;
  h->last_eps_mode = -1;  // the first captured J v sets epsilon's mode explicitly
  cudaGraph_t graph = nullptr;
  cudaError_t err = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
  const bool began = err == cudaSuccess;  // a begun capture is always ended below
  auto step = [&](cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; };
  if (err == cudaSuccess && key.basis == 32) {
    // FP32 basis, right preconditioning M^{-1} applied on the fly: z = M^{-1} v_j (FP64),
    // w = (J - sigma I) z (FP64), rounded into V32_{j+1}; x += M^{-1} (V32 y) at the end
    k_gm_cycle_init<<<1, 64, 0, h->stream>>>(D);
    step(kry_to_f32(h, W.r, n, W.dnorm, W.V32));
    for (int j = 0; j < m && err == cudaSuccess; ++j) {
      const float2* Vj = W.V32 + (size_t)j * n;
      float2* Vn = W.V32 + (size_t)(j + 1) * n;
      h->gate = D.flags;
      if (pc) step(pc_apply(h, nullptr, W.zt, Vj));
      else step(kry_to_f64(h, Vj, n, W.zt));
      step(jv_apply(h, W.zt, W.w, d2(sigma), eps_mode));
      step(kry_to_f32(h, W.w, n, nullptr, Vn));
      step(kry_dgks32(h, W.V32, j + 1, n, Vn, W.dh, W.dnorm, W.partial));
      h->gate = nullptr;
      k_gm_step<<<1, 32, 0, h->stream>>>(D, j);
      h->gate = D.flags;
      step(kry_scale32(h, Vn, n, W.dnorm));
      h->gate = nullptr;
    }
    k_gm_solve<<<1, 64, 0, h->stream>>>(D);
    step(kry_gemv32(h, W.V32, m, D.flags + 1, n, W.y, W.t));
    if (pc) step(pc_apply(h, W.t, W.zt));
    step(kry_axpby(h, make_double2(1.0, 0.0), pc ? W.zt : W.t, make_double2(1.0, 0.0), W.x, n));
    step(jv_apply(h, W.x, W.r, d2(sigma), eps_mode));
    step(kry_axpby(h, make_double2(1.0, 0.0), W.b, make_double2(-1.0, 0.0), W.r, n));
    step(launch_norm2(h, W.r, n, W.dnorm, 1));
  } else if (err == cudaSuccess) {
    k_gm_cycle_init<<<1, 64, 0, h->stream>>>(D);
    step(kry_scale(h, W.r, n, W.dnorm, W.V));
    for (int j = 0; j < m && err == cudaSuccess; ++j) {
      double2* Vj = W.V + (size_t)j * n;
      double2* Vn = W.V + (size_t)(j + 1) * n;
      double2* zj = pc ? W.Z + (size_t)j * n : Vj;
      h->gate = D.flags;
      if (pc) step(pc_apply(h, Vj, zj));
      step(jv_apply(h, zj, Vn, d2(sigma), eps_mode));
      // tiny vectors: the fused four-kernel CGS2 (launch latency dominates); otherwise the
      // selective form, which reads the basis half as often
      if (n < kSelectiveMinN) step(kry_cgs2(h, W.V, j + 1, n, Vn, W.dh, W.dnorm, W.partial));
      else step(kry_dgks(h, W.V, j + 1, n, Vn, W.dh, W.dnorm, W.partial));
      h->gate = nullptr;
      k_gm_step<<<1, 32, 0, h->stream>>>(D, j);
      h->gate = D.flags;
      step(kry_scale(h, Vn, n, W.dnorm, nullptr));
      h->gate = nullptr;
    }
    k_gm_solve<<<1, 64, 0, h->stream>>>(D);
    step(kry_gemv_add(h, pc ? W.Z : W.V, m, n, W.y, W.x, D.flags + 1));
    step(jv_apply(h, W.x, W.r, d2(sigma), eps_mode));
    step(kry_axpby(h, make_double2(1.0, 0.0), W.b, make_double2(-1.0, 0.0), W.r, n));
    step(launch_norm2(h, W.r, n, W.dnorm, 1));
  }
  if (began) {
    if (err == cudaSuccess) k_gm_report<<<1, 1, 0, h->stream>>>(D, rep);
    step(cudaGetLastError());
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (err == cudaSuccess) err = e2;
  }
  h->gate = nullptr;
  h->capturing = false;
  h->stream = saved_stream;
  h->stats = saved_stats;
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  ck(h, err, "GMRES cycle graph");
  h->gm_exec = exec;
  h->gm_key = key;
  return exec;
}

// (J - sigma I) x = b.  Returns the iteration count; sets *converged.
int gmres(StabHandle* h, cd sigma, const double2* b, double2* x, int eps_mode, bool* converged) {
  const long long n = h->n;
  const double tol = h->opts.gmres_tol;
  GmDev D;
  GmReport* d_rep;
  GmresWs W = gmres_ws(h, &D, &d_rep);
  cudaGraphExec_t exec = gm_graph(h, sigma, eps_mode, W, D, d_rep);
  ck(h, kry_copy(h, b, W.b, n), "copy b");
  ck(h, launch_norm2(h, W.b, n, W.dnorm, 1), "norm");
  const double bnorm = read_scalar(h, W.dnorm);
  *converged = false;
  if (!(bnorm < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: right-hand side is not finite");
  if (bnorm == 0.0) {
    ck(h, cudaMemsetAsync(x, 0, n * sizeof(double2), h->stream), "memset");
    *converged = true;
    return 0;
  }
  ck(h, cudaMemsetAsync(W.x, 0, n * sizeof(double2), h->stream), "memset");
  ck(h, kry_copy(h, W.b, W.r, n), "copy");
  k_gm_tol<<<1, 1, 0, h->stream>>>(D, tol);
  int total = 0;
  GmReport rep{};
  for (int cycle = 0; cycle < h->opts.gmres_max_restarts; ++cycle) {
    ck(h, cudaGraphLaunch(exec, h->stream), "GMRES cycle");
    ck(h, cudaMemcpyAsync(&rep, d_rep, sizeof(GmReport), cudaMemcpyDeviceToHost, h->stream), "report");
    ck(h, cudaStreamSynchronize(h->stream), "sync");
    total += rep.jend;
    h->stats.jv_calls += rep.jend + 1;
    if (rep.status) fail(h, STAB_ERR_NUMERIC, "GMRES: non-finite Krylov vector");
    if (!(rep.beta < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: non-finite residual");
    if (rep.beta <= tol * bnorm) { *converged = true; break; }
  }
  ck(h, kry_copy(h, W.x, x, n), "copy x");
  h->stats.gmres_iterations += total;
  h->stats.gmres_solves += 1;
  return total;
}

// ---------------------------------------------------------------------------
// Device-resident Hessenberg state of the implicit restart.
// ---------------------------------------------------------------------------
struct RestartWs {
  hd::zc *H, *T, *Z, *X, *Y, *Q, *theta, *sn, *Qc, *out_theta;
  double *cs, *est, *scal;  // scal: [conv count, fnorm, ||H||_F]
  int* order;
  hd::zc* coef;             // [beta_k, sigma_k]
};

size_t restart_ws_elems(int m, int k) {
  // complex elements: 7 m*m + 4 m + m*(k+1) + k + 2, plus doubles/ints packed as complex
  return (size_t)7 * m * m + 4 * m + (size_t)m * (k + 1) + k + 2 + (m + k + 4) + m;
}

RestartWs restart_ws(double2* base, int m, int k) {
  RestartWs w;
  hd::zc* p = (hd::zc*)base;
  w.H = p; p += (size_t)m * m;
  w.T = p; p += (size_t)m * m;
  w.Z = p; p += (size_t)m * m;
  w.X = p; p += (size_t)m * m;
  w.Y = p; p += (size_t)m * m;
  w.Q = p; p += (size_t)m * m;
  p += (size_t)m * m;  // spare
  w.theta = p; p += m;
  w.sn = p; p += m;
  w.out_theta = p; p += m;
  p += m;
  w.Qc = p; p += (size_t)m * (k + 1);
  w.coef = p; p += 2;
  double* d = (double*)p;
  w.cs = d; d += m;
  w.est = d; d += k;
  w.scal = d; d += 4;
  w.order = (int*)d;
  return w;
}

// H(0..j, j) = h;  H(j, j-1) = beta (when set)
__global__ void k_hcol(hd::zc* H, int m, int j, const double2* dh, const double* beta, int set_sub) {
  for (int i = threadIdx.x; i <= j; i += blockDim.x) H[i * m + j] = hd::mk(dh[i].x, dh[i].y);
  if (threadIdx.x == 0 && set_sub && j > 0) H[j * m + j - 1] = hd::mk(*beta, 0.0);
}

__global__ void k_hsub(hd::zc* H, int m, int j, const double* beta) { H[j * m + j - 1] = hd::mk(*beta, 0.0); }

__global__ void k_zero(hd::zc* H, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) H[i] = hd::mk(0.0);
}

// Spectrum of H_m, wanted/unwanted split, Ritz estimates (Eq. ritz_estimate);
// then either the wanted eigenvectors (finish = 1 or all converged) or the
// exact-shift sweeps and the coefficients of the basis update (Algorithm iram).
__global__ void k_restart(RestartWs w, int m, int k, double2 sg, double2 ta, double tol, const double* fnorm,
                          int finish) {
  if (threadIdx.x != 0) return;
  const hd::zc sigma = hd::mk(sg.x, sg.y), tau = hd::mk(ta.x, ta.y);
  if (hd::eig(m, w.H, w.theta, w.Y, w.T, w.Z, w.X) != 0) { w.scal[0] = -1.0; return; }
  for (int i = 0; i < m; ++i) w.order[i] = i;
  for (int i = 1; i < m; ++i) {  // insertion sort (stable) by the wanted order
    int v = w.order[i], j = i - 1;
    while (j >= 0 && hd::before(w.theta[v], w.theta[w.order[j]], sigma, tau)) { w.order[j + 1] = w.order[j]; --j; }
    w.order[j + 1] = v;
  }
  double hn = 0.0;
  for (int i = 0; i < m * m; ++i) hn += hd::abs2(w.H[i]);
  hn = sqrt(hn);
  const double fn = *fnorm;
  int conv = 0;
  for (int q = 0; q < k; ++q) {
    const int i = w.order[q];
    w.est[q] = fn * hd::zabs(w.Y[(m - 1) * m + i]);
    w.out_theta[q] = w.theta[i];
    if (w.est[q] <= fmax(2.220446049250313e-16 * hn, tol * hd::zabs(w.theta[i]))) ++conv;
  }
  w.scal[0] = conv;
  w.scal[1] = fn;
  w.scal[2] = hn;
  if (conv == k || finish) {
    for (int q = 0; q < k; ++q)
      for (int l = 0; l < m; ++l) w.Qc[q * m + l] = w.Y[l * m + w.order[q]];
    return;
  }
  for (int i = 0; i < m * m; ++i) w.Q[i] = hd::mk(0.0);
  for (int i = 0; i < m; ++i) w.Q[i * m + i] = hd::mk(1.0);
  for (int q = k; q < m; ++q) hd::shifted_qr(m, w.H, w.Q, w.theta[w.order[q]], w.cs, w.sn);
  w.coef[0] = w.H[k * m + k - 1];        // beta_k
  w.coef[1] = w.Q[(m - 1) * m + k - 1];  // sigma_k
  for (int j = 0; j <= k; ++j)
    for (int l = 0; l < m; ++l) w.Qc[j * m + l] = w.Q[l * m + j];
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c)
      if (r >= k || c >= k) w.H[r * m + c] = hd::mk(0.0);
}

// f = x * coef[0] + f * coef[1]  (coefficients in device memory)
__global__ void k_f_update(const double2* x, double2* f, long long n, const hd::zc* coef) {
  const hd::zc a = coef[0], b = coef[1];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 xv = x[i], fv = f[i];
    f[i] = make_double2(a.re * xv.x - a.im * xv.y + b.re * fv.x - b.im * fv.y,
                        a.re * xv.y + a.im * xv.x + b.re * fv.y + b.im * fv.x);
  }
}

// splitmix64 (Steele, Lea and Flood 2014): uniform [-1/2, 1/2) from the top 53 bits
void splitmix_start(unsigned long long seed, long long n, std::vector<double>& out) {
  out.resize(2 * (size_t)n);
  unsigned long long state = seed;
  double nrm = 0.0;
  for (long long i = 0; i < 2 * n; ++i) {
    state += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    out[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    nrm += out[i] * out[i];
  }
  nrm = std::sqrt(nrm);
  for (auto& v : out) v /= nrm;
}

}  // namespace

extern "C" stab_status stab_solve(stab_handle hh, double sr, double si, const void* b, void* x, int* iters) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  if (!b || !x) { h->err = "stab_solve: null vector"; return STAB_ERR_INVALID_ARG; }
  try {
    const cd sigma(sr, si);
    if (h->opts.precond == 1 && !(h->pvalid && h->psigma_re == sr && h->psigma_im == si))
      ck(h, pc_build(h, d2(sigma)), "preconditioner build");
    bool conv;
    int it = gmres(h, sigma, (const double2*)b, (double2*)x, h->opts.eps_mode, &conv);
    if (iters) *iters = it;
    if (!conv) { h->err = "stab_solve: GMRES restart limit reached"; return STAB_ERR_NOT_CONVERGED; }
    return STAB_OK;
  } catch (Fail& f) {
    return f.st;
  }
}

extern "C" stab_status stab_orthogonalize(stab_handle hh, const void* V, int k, void* w, double* hcoef, double* norm) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  if ((k > 0 && !V) || !w || k < 0) { h->err = "stab_orthogonalize: bad arguments"; return STAB_ERR_INVALID_ARG; }
  try {
    const long long n = h->n;
    const size_t part = (size_t)kry_partial_elems(n, k);
    double2* ws = ensure(h, &h->d_ir, &h->ir_elems, part + 2 * (size_t)std::max(k, 1) + 2);
    double2* dh = ws + part;
    double* dn = (double*)(dh + 2 * std::max(k, 1));
    ck(h, kry_cgs2(h, (const double2*)V, k, n, (double2*)w, dh, dn, ws), "CGS2");
    if (hcoef && k > 0) ck(h, cudaMemcpyAsync(hcoef, dh, sizeof(double2) * k, cudaMemcpyDeviceToHost, h->stream), "copy");
    double nv = 0.0;
    ck(h, cudaMemcpyAsync(&nv, dn, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy");
    ck(h, cudaStreamSynchronize(h->stream), "sync");
    if (norm) *norm = nv;
    return STAB_OK;
  } catch (Fail& f) {
    return f.st;
  }
}

extern "C" stab_status stab_jv_batch_orthogonalize(stab_jv_batch B, const void* const* V, const int* k, void* const* w,
                                                   double* hcoef, double* norms) {
  if (!B) return STAB_ERR_INVALID_ARG;
  const int count = (int)B->hs.size();
  if (!V || !k || !w) {
    B->err = "stab_jv_batch_orthogonalize: null argument list";
    return STAB_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i)
    if (!V[i] || !w[i] || k[i] < 1 || k[i] > 1536) {
      B->err = "stab_jv_batch_orthogonalize: instance " + std::to_string(i) + " needs V, w and 1 <= k <= 1536";
      return STAB_ERR_INVALID_ARG;
    }
  std::vector<CgsJob> jobs;
  std::vector<const double2*> dhs;
  std::vector<const double*> dns;
  for (int i = 0; i < count; ++i) {
    StabHandle* h = B->hs[i];
    try {  // the scratch of stab_orthogonalize, allocated on the handle's stream
      const long long n = h->n;
      const size_t part = (size_t)kry_partial_elems(n, k[i]);
      double2* ws = ensure(h, &h->d_ir, &h->ir_elems, part + 2 * (size_t)k[i] + 2);
      double2* dh = ws + part;
      double* dn = (double*)(dh + 2 * k[i]);
      ck(h, cudaStreamSynchronize(h->stream), "sync");  // the allocation is usable on the batch's stream
      jobs.push_back(CgsJob{(const double2*)V[i], k[i], n, (double2*)w[i], dh, dn, ws});
      dhs.push_back(dh);
      dns.push_back(dn);
    } catch (Fail& f) {
      B->err = "stab_jv_batch_orthogonalize: instance " + std::to_string(i) + ": " + h->err;
      return f.st;
    }
  }
  cudaError_t e = kry_cgs2_batch(B, jobs);
  size_t off = 0;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    if (hcoef) e = cudaMemcpyAsync(hcoef + 2 * off, dhs[i], sizeof(double2) * k[i], cudaMemcpyDeviceToHost, B->stream);
    if (norms && e == cudaSuccess) e = cudaMemcpyAsync(norms + i, dns[i], sizeof(double), cudaMemcpyDeviceToHost, B->stream);
    off += (size_t)k[i];
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
  if (e != cudaSuccess) {
    B->err = std::string("stab_jv_batch_orthogonalize: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA;
  }
  return STAB_OK;
}

extern "C" stab_status stab_eigs(stab_handle hh, double sr, double si, double tr, double ti, int nev, int ncv,
                                 double tol, const void* v0, double* lambda, void* vecs, double* resid, int* nconv,
                                 stab_stats* stats) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  if (nev < 1 || ncv <= nev || ncv > 512 || ncv > h->n || !(tol > 0) || !lambda || !nconv) {
    h->err = "stab_eigs: need 1 <= nev < ncv <= min(n, 512), tol > 0, lambda and nconv";
    return STAB_ERR_INVALID_ARG;
  }
  const auto t_start = std::chrono::steady_clock::now();
  const stab_stats s0 = h->stats;
  const cd sigma(sr, si), tau(tr, ti);
  const int k = nev, m = ncv;
  const long long n = h->n;
  stab_status result = STAB_OK;
  try {
    if (h->opts.precond == 1 && !(h->pvalid && h->psigma_re == sr && h->psigma_im == si)) {
      auto tp = std::chrono::steady_clock::now();
      ck(h, pc_build(h, d2(sigma)), "preconditioner build");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
      h->stats.seconds_precond += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
    }
    // IRAM workspace: V (m n), f (n), x (n), tmp ((k+1) n), partials, dh, scalars, restart state
    const size_t part = (size_t)kry_partial_elems(n, m);
    const size_t rws = restart_ws_elems(m, k);
    const size_t need = (size_t)m * n + 2 * (size_t)n + (size_t)(k + 1) * n + part + 2 * m + 4 + rws;
    double2* base = ensure(h, &h->d_ir, &h->ir_elems, need);
    double2* V = base;
    double2* f = V + (size_t)m * n;
    double2* xw = f + n;
    double2* tmp = xw + n;
    double2* partial = tmp + (size_t)(k + 1) * n;
    double2* dh = partial + part;
    double* dn = (double*)(dh + 2 * m);
    RestartWs RW = restart_ws(dh + 2 * m + 4, m, k);
    const double2* dQ = (const double2*)RW.Qc;
    // start vector
    if (v0) ck(h, kry_copy(h, (const double2*)v0, f, n), "copy v0");
    else {
      std::vector<double> sv;
      splitmix_start(h->opts.seed, n, sv);
      ck(h, cudaMemcpyAsync(f, sv.data(), sizeof(double) * sv.size(), cudaMemcpyHostToDevice, h->stream), "copy start");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
    }
    k_zero<<<1, 256, 0, h->stream>>>(RW.H, m * m);
    std::vector<double> ritz(2 * k + k + 4);
    int j0 = 0;
    bool first = true;
    int conv_count = 0;
    std::vector<cd> theta_w(k);
    for (int restart = 0;; ++restart) {
      for (int j = j0; j < m; ++j) {
        ck(h, launch_norm2(h, f, n, dn, 1), "norm");
        const double beta = read_scalar(h, dn);
        if (!(beta < INFINITY)) fail(h, STAB_ERR_NUMERIC, "IRAM: non-finite residual vector");
        if (beta == 0.0) fail(h, STAB_ERR_BREAKDOWN, "IRAM: Arnoldi breakdown (invariant subspace)");
        // H(j, j-1) = beta from the device norm; the column H(0..j, j) follows the orthogonalisation
        double2* Vj = V + (size_t)j * n;
        if (!first || j > 0) k_hsub<<<1, 1, 0, h->stream>>>(RW.H, m, j, dn);
        ck(h, kry_scale(h, f, n, dn, Vj), "scale");
        // w = C v_j: b = (J - tau I) v_j, then (J - sigma I) x = b
        ck(h, jv_apply(h, Vj, xw, d2(tau), h->opts.eps_mode), "J v");
        bool gconv;
        gmres(h, sigma, xw, f, h->opts.eps_mode, &gconv);
        if (!gconv) result = STAB_ERR_NOT_CONVERGED;
        ck(h, kry_cgs2(h, V, j + 1, n, f, dh, dn, partial), "CGS2");
        k_hcol<<<1, 64, 0, h->stream>>>(RW.H, m, j, dh, dn, 0);
        h->stats.arnoldi_steps++;
      }
      first = false;
      const int finish = restart >= h->opts.max_restarts;
      k_restart<<<1, 32, 0, h->stream>>>(RW, m, k, d2(sigma), d2(tau), tol, dn, finish);
      ck(h, cudaGetLastError(), "restart kernel");
      ck(h, cudaMemcpyAsync(ritz.data(), RW.out_theta, sizeof(double2) * k, cudaMemcpyDeviceToHost, h->stream), "copy");
      ck(h, cudaMemcpyAsync(ritz.data() + 2 * k, RW.est, sizeof(double) * (k + 4), cudaMemcpyDeviceToHost, h->stream),
         "copy");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
      const double* scal = ritz.data() + 3 * k;
      if (scal[0] < 0) fail(h, STAB_ERR_NUMERIC, "IRAM: Hessenberg QR failed");
      conv_count = (int)scal[0];
      for (int q = 0; q < k; ++q) theta_w[q] = cd(ritz[2 * q], ritz[2 * q + 1]);
      if (conv_count == k || finish) {
        if (conv_count < k) { result = STAB_ERR_NOT_CONVERGED; h->err = "stab_eigs: IRAM restart limit reached"; }
        break;
      }
      h->stats.restarts++;
      // tmp = V Q[:, 0:k+1];  f = tmp_k beta_k + f sigma_k;  V[:, 0:k] = tmp[:, 0:k]
      ck(h, kry_update_basis(h, V, m, k + 1, n, dQ, tmp), "V Q");
      k_f_update<<<1024, 256, 0, h->stream>>>(tmp + (size_t)k * n, f, n, RW.coef);
      ck(h, cudaMemcpyAsync(V, tmp, sizeof(double2) * (size_t)k * n, cudaMemcpyDeviceToDevice, h->stream), "copy V");
      j0 = k;
    }
    // eigenpairs: x_q = V y_q (the wanted Ritz vectors are in Qc), lambda_q = (sigma theta - tau)/(theta - 1)
    double2* X = tmp;  // k vectors (tmp holds k + 1)
    ck(h, kry_update_basis(h, V, m, k, n, dQ, X), "V Y");
    for (int q = 0; q < k; ++q) {
      const cd t = theta_w[q];
      const cd lam = (sigma * t - tau) / (t - 1.0);
      lambda[2 * q] = lam.real();
      lambda[2 * q + 1] = lam.imag();
      double2* xq = X + (size_t)q * n;
      ck(h, launch_norm2(h, xq, n, dn, 1), "norm");
      ck(h, kry_scale(h, xq, n, dn, nullptr), "normalise");
      if (resid) {  // true residual with the exact tangent
        ck(h, jv_apply(h, xq, xw, d2(lam), 2), "J x");
        ck(h, launch_norm2(h, xw, n, dn, 1), "norm");
        resid[q] = read_scalar(h, dn);
      }
      if (vecs) ck(h, kry_copy(h, xq, (double2*)vecs + (size_t)q * n, n), "copy vector");
    }
    ck(h, cudaStreamSynchronize(h->stream), "sync");
    *nconv = conv_count;
  } catch (Fail& fl) {
    result = fl.st;
  }
  h->stats.seconds_total += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  if (stats) {
    stab_stats d = h->stats;
    d.jv_calls -= s0.jv_calls;
    d.gmres_iterations -= s0.gmres_iterations;
    d.gmres_solves -= s0.gmres_solves;
    d.arnoldi_steps -= s0.arnoldi_steps;
    d.restarts -= s0.restarts;
    d.precond_builds -= s0.precond_builds;
    d.seconds_total -= s0.seconds_total;
    d.seconds_precond -= s0.seconds_precond;
    *stats = d;
  }
  return result;
}
