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


constexpr int kMaxGmresM = 200;  // stab_create rejects larger gmres_m
constexpr long long kSelectiveMinN = 16384;  // unknowns from which GMRES uses selective reorthogonalisation

// Device-resident least-squares state of one GMRES cycle: the rotated
// Hessenberg columns R (m x m, row-major), the rotated right-hand side g,
// the Givens rotations (cs, sn), flags [done, jend, status] and the scalars
// [tol ||b||, |g_{j+1}|, beta at the cycle start, ||dz|| (LGMRES)].
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

// GMRES workspace layout (complex elements).  FP64 basis: V, Z (flexible).
// FP32 basis: V32, and FP64 work vectors w (J z), zt (preconditioned
// direction or correction) and t (V32 y).  Nested inner solver (FP64 outer
// flexible GMRES): the inner FP32 basis V32 with w, zt, t, and the inner
// cycle's least-squares state Din.
struct GmresWs {
  double2 *V, *Z, *r, *b, *x, *partial, *dh, *y;
  double* dnorm;
  float2* V32;
  double2 *w, *zt, *t;
  double2 *AZ, *AAZ, *dz;  // LGMRES: augmentation vectors z_a and A z_a (newest first), the cycle's correction
  GmDev Din;               // nested inner GMRES (gmres_inner_m > 0)
  int mi = 0;
};

struct GmReport {  // read by the host once per cycle
  double beta;     // ||b - A x|| after the cycle
  double znorm;    // LGMRES: ||x_new - x_old|| of the cycle (0: no augmentation vector stored)
  double inner;    // nested inner solver: inner iterations (J v products) of the cycle
  int jend;        // iterations performed in the cycle
  int status;      // 0, or 1 when a Krylov quantity was not finite
};

GmresWs gmres_ws(StabHandle* h, GmDev* D, GmReport** rep) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond != 0;
  const bool b32 = h->opts.gmres_basis_prec == 32;
  const int lgk = b32 ? 0 : h->opts.lgmres_k;
  const int mi = b32 ? 0 : h->opts.gmres_inner_m;
  const bool flex = pc || lgk > 0 || mi > 0;  // the directions Z_j are stored
  const int mp = std::max(m, mi);
  const size_t part = (size_t)std::max(kry_partial_elems(n, mp + 1), kry_dgks_partial_elems(n, mp + 1));
  const size_t small = (size_t)m * m + (m + 1) + m + (m + 1) / 2 + 1 + 4 + 4;
  const size_t small_in = mi > 0 ? (size_t)mi * mi + (mi + 1) + mi + (mi + 1) / 2 + 1 + 4 + 2 * (mi + 1) + (mi + 1) + 4
                                 : 0;
  const size_t basis = b32 ? ((size_t)(m + 1) * n + 1) / 2 : (size_t)(m + 1) * n + (flex ? (size_t)m * n : 0);
  const size_t inner = mi > 0 ? ((size_t)(mi + 1) * n + 1) / 2 + 3 * (size_t)n : 0;
  const size_t work = (b32 ? 6 * (size_t)n : 3 * (size_t)n + (lgk > 0 ? (2 * (size_t)lgk + 1) * n : 0)) + inner;
  size_t need = basis + work + part + 2 * (m + 1) + (m + 1) + 4 + small + small_in;
  double2* base = ensure(h, &h->d_gm, &h->gm_elems, need);
  GmresWs w{};
  if (b32) {
    w.V32 = (float2*)base;
  } else {
    w.V = base;
    w.Z = flex ? base + (size_t)(m + 1) * n : nullptr;
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
  if (lgk > 0) {
    w.AZ = q;
    w.AAZ = q + (size_t)lgk * n;
    w.dz = q + 2 * (size_t)lgk * n;
    q += (2 * (size_t)lgk + 1) * n;
  }
  if (mi > 0) {
    w.w = q;
    w.zt = q + n;
    w.t = q + 2 * n;
    w.V32 = (float2*)(q + 3 * n);
    q += 3 * (size_t)n + ((size_t)(mi + 1) * n + 1) / 2;
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
  D->sc = (double*)p; p += 2;        // 4 doubles
  *rep = (GmReport*)p; p += 2;       // 24 bytes
  D->dh = w.dh;
  D->dnorm = w.dnorm;
  D->y = w.y;
  D->m = m;
  if (mi > 0) {  // the inner cycle's own least-squares state, coefficients, norm and solution
    GmDev& I = w.Din;
    I.R = (hd::zc*)p; p += (size_t)mi * mi;
    I.g = (hd::zc*)p; p += mi + 1;
    I.sn = (hd::zc*)p; p += mi;
    I.cs = (double*)p; p += (mi + 1) / 2 + 1;
    I.flags = (int*)p; p += 1;
    I.sc = (double*)p; p += 2;
    I.dh = p; p += 2 * (mi + 1);
    I.y = p; p += mi + 1;
    I.dnorm = (double*)p; p += 2;
    I.m = mi;
    w.mi = mi;
  }
  return w;
}

double read_scalar(StabHandle* h, const double* d) {
  double v;
  ck(h, cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read scalar");
  ck(h, cudaStreamSynchronize(h->stream), "sync");
  return v;
}

__global__ void k_gm_tol(GmDev d, double tol) { d.sc[0] = tol * (*d.dnorm); }

// start of a cycle: g = (beta, 0, ...), beta = ||r|| (in dnorm, kept in sc[2])
__global__ void k_gm_cycle_init(GmDev d) {
  if (threadIdx.x == 0) {
    d.flags[0] = 0;
    d.flags[1] = 0;
    d.flags[2] = 0;
    d.sc[2] = *d.dnorm;
    d.sc[3] = 0.0;
  }
  for (int i = threadIdx.x; i <= d.m; i += blockDim.x) d.g[i] = hd::mk(i == 0 ? *d.dnorm : 0.0);
}

__device__ __forceinline__ bool finite_zc(hd::zc z) { return fabs(z.re) < INFINITY && fabs(z.im) < INFINITY; }

// Arnoldi column j (h_0..h_j from CGS2, h_{j+1} = ||w||): previous rotations,
// the new rotation that annihilates h_{j+1}, the rotated right-hand side and
// the convergence test |g_{j+1}| <= tol ||b|| (or w = 0).  One warp: the
// column and the rotations are staged in shared memory by all lanes, the
// rotation chain runs on lane 0.
__device__ __forceinline__ void gm_step_body(const GmDev& d, int j) {
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

__global__ void k_gm_step(GmDev d, int j) { gm_step_body(d, j); }

// y = R^{-1} g over the jend columns of the cycle, by columns: y_i from the
// diagonal, then every thread removes y_i's contribution from its rows.
__device__ __forceinline__ void gm_solve_body(const GmDev& d) {
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

__global__ void k_gm_solve(GmDev d) { gm_solve_body(d); }

__global__ void k_gm_report(GmDev d, GmReport* rep, const double* inner_tally) {
  rep->beta = *d.dnorm;
  rep->znorm = d.sc[3];
  rep->inner = inner_tally ? *inner_tally : 0.0;
  rep->jend = d.flags[1];
  rep->status = d.flags[2];
}

// Nested inner GMRES of one outer step: (J - sigma I) z = v_j from z = 0 with
// ||v_j|| = 1, gated by the outer cycle (an outer cycle that has converged
// skips its remaining inner solves); tol_in relative to ||v_j||.
__global__ void k_gm_inner_init(GmDev in, const int* outer_flags, double tol_in) {
  if (threadIdx.x == 0) {
    in.flags[0] = outer_flags[0];
    in.flags[1] = 0;
    in.flags[2] = 0;
    *const_cast<double*>(in.dnorm) = 1.0;
    in.sc[0] = tol_in;
  }
  for (int i = threadIdx.x; i <= in.m; i += blockDim.x) in.g[i] = hd::mk(i == 0 ? 1.0 : 0.0);
}

// the inner iterations of a cycle, tallied in the inner state's sc[3]
__global__ void k_gm_inner_reset(GmDev in) { in.sc[3] = 0.0; }
__global__ void k_gm_inner_tally(GmDev in) { in.sc[3] += in.flags[1]; }

// LGMRES: the newest augmentation pair from the cycle's correction dz and the
// residuals before (beta_0 V_0) and after (r) it: z = dz / ||dz||,
// A z = (beta_0 V_0 - r) / ||dz||; zeros when dz = 0 (the host then drops
// the stored pairs).
__global__ void k_lg_store(double2* __restrict__ z, double2* __restrict__ az, const double2* __restrict__ dz,
                           const double2* __restrict__ v0, const double2* __restrict__ r, const double* sc,
                           long long n) {
  const double b0 = sc[2], zn = sc[3];
  const double s = zn > 0.0 ? 1.0 / zn : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 d = dz[i], v = v0[i], q = r[i];
    z[i] = make_double2(d.x * s, d.y * s);
    az[i] = make_double2((b0 * v.x - q.x) * s, (b0 * v.y - q.y) * s);
  }
}

// One GMRES cycle as a CUDA graph: V_0 = r / beta; m Arnoldi steps, each
// (right preconditioner, J v - sigma v, Gram-Schmidt with selective
// reorthogonalisation, Givens update, scaling) gated
// on the device flag that the Givens update raises at convergence; the
// least-squares solve, x += Z y (V y), and the true residual r = b - A x with
// its norm.  Captured once per handle, shift and workspace, replayed for
// every cycle of every solve: the host only reads the report once per cycle.
cudaGraphExec_t gm_graph(StabHandle* h, cd sigma, int eps_mode, const GmresWs& W, const GmDev& D, GmReport* rep,
                         int naug) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond != 0;
  const int lgk = h->opts.gmres_basis_prec == 32 ? 0 : h->opts.lgmres_k;
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
  key.lgk = lgk;
  key.naug = naug;
  key.mi = W.mi;
  cudaGraphExec_t& slot = h->gm_exec[naug];
  GmGraphKey& slot_key = h->gm_key[naug];
  if (slot && key == slot_key) return slot;
  if (slot) {
    cudaGraphExecDestroy(slot);
    slot = nullptr;
    slot_key.valid = false;
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
    // LGMRES: the last naug of the m steps take the stored augmentation pairs (z_a, A z_a) instead of
    // a preconditioned Krylov direction and its J v
    const int mi = W.mi;
    const bool flex = pc || lgk > 0 || mi > 0;
    const int nkry = m - naug;
    k_gm_cycle_init<<<1, 64, 0, h->stream>>>(D);
    if (mi > 0) k_gm_inner_reset<<<1, 1, 0, h->stream>>>(W.Din);
    step(kry_scale(h, W.r, n, W.dnorm, W.V));
    for (int j = 0; j < m && err == cudaSuccess; ++j) {
      double2* Vj = W.V + (size_t)j * n;
      double2* Vn = W.V + (size_t)(j + 1) * n;
      double2* zj = flex ? W.Z + (size_t)j * n : Vj;
      h->gate = D.flags;
      if (mi > 0) {
        // nested: z_j = the inner FP32-basis GMRES(mi) approximation of (J - sigma I)^{-1} v_j (right
        // preconditioned with the block inverses), the same steps as the FP32-basis cycle below
        const GmDev& I = W.Din;
        h->gate = nullptr;
        k_gm_inner_init<<<1, 64, 0, h->stream>>>(I, D.flags, h->opts.gmres_inner_tol);
        h->gate = I.flags;
        step(kry_to_f32(h, Vj, n, nullptr, W.V32));
        for (int i = 0; i < mi && err == cudaSuccess; ++i) {
          const float2* Vi = W.V32 + (size_t)i * n;
          float2* Vi1 = W.V32 + (size_t)(i + 1) * n;
          h->gate = I.flags;
          if (pc) step(pc_apply(h, nullptr, W.zt, Vi));
          else step(kry_to_f64(h, Vi, n, W.zt));
          step(jv_apply(h, W.zt, W.w, d2(sigma), eps_mode));
          step(kry_to_f32(h, W.w, n, nullptr, Vi1));
          step(kry_dgks32(h, W.V32, i + 1, n, Vi1, const_cast<double2*>(I.dh), const_cast<double*>(I.dnorm),
                          W.partial));
          h->gate = nullptr;
          k_gm_step<<<1, 32, 0, h->stream>>>(I, i);
          h->gate = I.flags;
          step(kry_scale32(h, Vi1, n, I.dnorm));
        }
        h->gate = nullptr;
        k_gm_solve<<<1, 64, 0, h->stream>>>(I);
        k_gm_inner_tally<<<1, 1, 0, h->stream>>>(I);
        step(kry_gemv32(h, W.V32, mi, I.flags + 1, n, I.y, W.t));
        h->gate = D.flags;
        if (pc) step(pc_apply(h, W.t, zj));
        else step(kry_copy(h, W.t, zj, n));
        step(jv_apply(h, zj, Vn, d2(sigma), eps_mode));
      } else if (j < nkry) {
        if (pc) step(pc_apply(h, Vj, zj));
        else if (flex) step(kry_copy(h, Vj, zj, n));
        step(jv_apply(h, zj, Vn, d2(sigma), eps_mode));
      } else {
        const size_t a = (size_t)(j - nkry);
        step(kry_copy(h, W.AZ + a * n, zj, n));
        step(kry_copy(h, W.AAZ + a * n, Vn, n));
      }
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
    if (lgk > 0) {
      // dz = Z y; x += dz; r = b - A x; store (dz, r_old - r) / ||dz|| as the newest pair after
      // moving the older ones one slot down
      step(cudaMemsetAsync(W.dz, 0, (size_t)n * sizeof(double2), h->stream));
      step(kry_gemv_add(h, W.Z, m, n, W.y, W.dz, D.flags + 1));
      step(kry_axpby(h, make_double2(1.0, 0.0), W.dz, make_double2(1.0, 0.0), W.x, n));
      step(jv_apply(h, W.x, W.r, d2(sigma), eps_mode));
      step(kry_axpby(h, make_double2(1.0, 0.0), W.b, make_double2(-1.0, 0.0), W.r, n));
      step(launch_norm2(h, W.dz, n, D.sc + 3, 1));
      for (int a = lgk - 1; a >= 1; --a) {
        step(kry_copy(h, W.AZ + (size_t)(a - 1) * n, W.AZ + (size_t)a * n, n));
        step(kry_copy(h, W.AAZ + (size_t)(a - 1) * n, W.AAZ + (size_t)a * n, n));
      }
      const int thr = 256;
      const long long nb = std::min<long long>((n + thr - 1) / thr, 152LL * 8);
      k_lg_store<<<(unsigned)nb, thr, 0, h->stream>>>(W.AZ, W.AAZ, W.dz, W.V, W.r, D.sc, n);
      step(cudaGetLastError());
    } else {
      step(kry_gemv_add(h, flex ? W.Z : W.V, m, n, W.y, W.x, D.flags + 1));
      step(jv_apply(h, W.x, W.r, d2(sigma), eps_mode));
      step(kry_axpby(h, make_double2(1.0, 0.0), W.b, make_double2(-1.0, 0.0), W.r, n));
    }
    step(launch_norm2(h, W.r, n, W.dnorm, 1));
  }
  if (began) {
    if (err == cudaSuccess) k_gm_report<<<1, 1, 0, h->stream>>>(D, rep, W.mi > 0 ? W.Din.sc + 3 : nullptr);
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
  slot = exec;
  slot_key = key;
  return exec;
}

// (J - sigma I) x = b.  Returns the iteration count; sets *converged.
int gmres(StabHandle* h, cd sigma, const double2* b, double2* x, int eps_mode, bool* converged) {
  const long long n = h->n;
  const double tol = h->opts.gmres_tol;
  GmDev D;
  GmReport* d_rep;
  GmresWs W = gmres_ws(h, &D, &d_rep);
  const int m = h->opts.gmres_m;
  const int lgk = h->opts.gmres_basis_prec == 32 ? 0 : h->opts.lgmres_k;
  int naug = 0;  // LGMRES augmentation pairs stored by earlier cycles of this solve
  cudaGraphExec_t exec = gm_graph(h, sigma, eps_mode, W, D, d_rep, 0);
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
    if (lgk > 0) exec = gm_graph(h, sigma, eps_mode, W, D, d_rep, naug);
    ck(h, cudaGraphLaunch(exec, h->stream), "GMRES cycle");
    ck(h, cudaMemcpyAsync(&rep, d_rep, sizeof(GmReport), cudaMemcpyDeviceToHost, h->stream), "report");
    ck(h, cudaStreamSynchronize(h->stream), "sync");
    total += rep.jend;
    h->stats.jv_calls += std::min(rep.jend, m - naug) + 1 + (long long)rep.inner;  // augmentation steps take
                                                                                     // no J v; inner steps one
    if (lgk > 0) naug = rep.znorm > 0.0 ? std::min(naug + 1, lgk) : 0;
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
__device__ void restart_body(const RestartWs& w, int m, int k, double2 sg, double2 ta, double tol, const double* fnorm,
                             int finish) {
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

__global__ void k_restart(RestartWs w, int m, int k, double2 sg, double2 ta, double tol, const double* fnorm,
                          int finish) {
  if (threadIdx.x != 0) return;
  restart_body(w, m, k, sg, ta, tol, fnorm, finish);
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
    if (h->opts.precond != 0 && !(h->pvalid && h->psigma_re == sr && h->psigma_im == si))
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
    if (h->opts.precond != 0 && !(h->pvalid && h->psigma_re == sr && h->psigma_im == si)) {
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

// ===========================================================================
// Solver-level batching (stab_jv_batch_solve, stab_jv_batch_eigs): the GMRES
// cycles and the Arnoldi steps of every instance of a batch advance in
// lockstep, each phase one launch for all instances (the stab_jv_batch
// kernels, whose items carry per-instance device gates).  An instance that
// has converged, or whose cycle ended early, is skipped through its gate
// without a host round trip; the host reads one report per cycle for all
// instances.  The parameter images of every phase are built once per solve
// and copied to the device once.
// ===========================================================================
namespace {

struct VecItem {  // y = x / *norm (op 0) or y = a x + b y (op 1)
  const double2* x;
  double2* y;
  const double* norm;
  const int* gate;
  long long n;
  double2 a, b;
  int op, pad;
};
static_assert(sizeof(VecItem) % 8 == 0, "items are read as 8-byte words");
constexpr int kVecScale = 0, kVecAxpby = 1;

struct GemvItem {  // x += V[:, 0:min(k, *kdev)] y
  const double2* V;
  const double2* y;
  double2* x;
  const int* kdev;
  const int* gate;
  long long n;
  int k, pad;
};
static_assert(sizeof(GemvItem) % 8 == 0, "items are read as 8-byte words");

struct HItem {  // Hessenberg entries of an Arnoldi step: H(j, j-1) = *dn (op 0) or H(0..j, j) = dh (op 1)
  hd::zc* H;
  const double2* dh;
  const double* dn;
  const int* gate;
  int m, j, op, pad;
};
static_assert(sizeof(HItem) % 8 == 0, "items are read as 8-byte words");

struct RsItem {  // implicit restart of one instance (restart_body)
  RestartWs w;
  double2 sg, ta;
  double tol;
  const double* fnorm;
  const int* gate;
  int m, k, finish, pad;
};
static_assert(sizeof(RsItem) % 8 == 0, "items are read as 8-byte words");

__device__ __forceinline__ int find_item(const int* __restrict__ start, int count, unsigned b) {
  int lo = 0, hi = count - 1;  // largest i with start[i] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the arithmetic of k_scale_inv and k_axpby, per item
__global__ void k_bvec(const VecItem* __restrict__ items, const int* __restrict__ start, int count) {
  const int i = find_item(start, count, blockIdx.x);
  const VecItem it = items[i];
  if (it.gate && *it.gate) return;
  const long long s0 = __ldg(start + i), nb = __ldg(start + i + 1) - s0;
  const long long b0 = (long long)blockIdx.x - s0;
  if (it.op == kVecScale) {
    const double s = 1.0 / *it.norm;
    for (long long q = b0 * blockDim.x + threadIdx.x; q < it.n; q += nb * blockDim.x) {
      double2 v = it.x[q];
      it.y[q] = make_double2(v.x * s, v.y * s);
    }
  } else {
    const double2 a = it.a, b = it.b;
    for (long long q = b0 * blockDim.x + threadIdx.x; q < it.n; q += nb * blockDim.x) {
      double2 xv = it.x[q], yv = it.y[q];
      it.y[q] = make_double2(a.x * xv.x - a.y * xv.y + b.x * yv.x - b.y * yv.y,
                             a.x * xv.y + a.y * xv.x + b.x * yv.y + b.y * yv.x);
    }
  }
}

// the arithmetic of k_gemv (sign +1), per item
__global__ void __launch_bounds__(256) k_bgemv(const GemvItem* __restrict__ items, const int* __restrict__ start,
                                               int count) {
  __shared__ double2 hs[kMaxGmresM + 1];
  const int i = find_item(start, count, blockIdx.x);
  const GemvItem it = items[i];
  if (it.gate && *it.gate) return;
  int k = it.k;
  if (it.kdev) k = min(k, *it.kdev);
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = it.y[j];
  __syncthreads();
  const long long s0 = __ldg(start + i), nb = __ldg(start + i + 1) - s0;
  const long long b0 = (long long)blockIdx.x - s0;
  const long long n = it.n;
  for (long long q = b0 * blockDim.x + threadIdx.x; q < n; q += nb * blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < k; ++j) {
      double2 a = it.V[(long long)j * n + q], c = hs[j];
      ar = fma(a.x, c.x, fma(-a.y, c.y, ar));
      ai = fma(a.x, c.y, fma(a.y, c.x, ai));
    }
    double2 xv = it.x[q];
    it.x[q] = make_double2(fma(1.0, ar, xv.x), fma(1.0, ai, xv.y));
  }
}

__global__ void k_bhess(const HItem* __restrict__ items, int count) {
  if ((int)blockIdx.x >= count) return;
  const HItem it = items[blockIdx.x];
  if (it.gate && *it.gate) return;
  if (it.op == 0) {
    if (threadIdx.x == 0) it.H[it.j * it.m + it.j - 1] = hd::mk(*it.dn, 0.0);
  } else {
    for (int i = threadIdx.x; i <= it.j; i += blockDim.x) it.H[i * it.m + it.j] = hd::mk(it.dh[i].x, it.dh[i].y);
  }
}

__global__ void k_brestart(const RsItem* __restrict__ items, int count) {
  if ((int)blockIdx.x >= count || threadIdx.x != 0) return;
  const RsItem it = items[blockIdx.x];
  if (it.gate && *it.gate) return;
  restart_body(it.w, it.m, it.k, it.sg, it.ta, it.tol, it.fnorm, it.finish);
}

// GMRES cycle state of every instance: flags[3] = the solve has converged (or
// the instance does not take part), which gates the whole cycle; flags[0]
// gates the Arnoldi steps as in the single-problem cycle.
__global__ void k_bgm_init(const GmDev* __restrict__ devs) {
  const GmDev d = devs[blockIdx.x];
  if (d.flags[3]) {
    if (threadIdx.x == 0) { d.flags[0] = 1; d.flags[1] = 0; d.flags[2] = 0; }
    return;
  }
  if (threadIdx.x == 0) {
    d.flags[0] = 0;
    d.flags[1] = 0;
    d.flags[2] = 0;
    d.sc[2] = *d.dnorm;
    d.sc[3] = 0.0;
  }
  for (int i = threadIdx.x; i <= d.m; i += blockDim.x) d.g[i] = hd::mk(i == 0 ? *d.dnorm : 0.0);
}

__global__ void k_bgm_step(const GmDev* __restrict__ devs, int j) {
  const GmDev d = devs[blockIdx.x];
  if (j >= d.m) return;
  gm_step_body(d, j);
}

__global__ void k_bgm_solve(const GmDev* __restrict__ devs) {
  const GmDev d = devs[blockIdx.x];
  if (d.flags[3]) return;
  gm_solve_body(d);
}

// report of the cycle; an instance whose true residual meets its tolerance
// (or that met a non-finite value) is done
__global__ void k_bgm_report(const GmDev* __restrict__ devs, GmReport* reps) {
  if (threadIdx.x != 0) return;
  const GmDev d = devs[blockIdx.x];
  GmReport r;
  r.beta = *d.dnorm;
  r.znorm = 0.0;
  r.jend = d.flags[1];
  r.status = d.flags[2];
  reps[blockIdx.x] = r;
  if (!d.flags[3] && (r.status || !(r.beta > d.sc[0]))) d.flags[3] = 1;
}

__global__ void k_bgm_begin(const GmDev* __restrict__ devs, const int* __restrict__ done, double tol_unused) {
  if (threadIdx.x != 0) return;
  const GmDev d = devs[blockIdx.x];
  d.flags[3] = done[blockIdx.x];
}

__global__ void k_gather(const double* const* __restrict__ src, double* out, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) out[i] = *src[i];
}

// elementwise / gemv item blocks: the grid of the single launch (grid_n), capped
template <class T>
int vec_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(b, 152LL * 8));
}

// Device copy of a parameter image plus small per-instance arrays, freed in stream order.
struct DevImage {
  void* d = nullptr;
  cudaStream_t st = nullptr;
  ~DevImage() {
    if (d) cudaFreeAsync(d, st);
  }
};

cudaError_t upload(DevImage& D, int device, cudaStream_t st, const BatchImage& im) {
  D.st = st;
  cudaError_t e = dev_alloc_stream(device, st, &D.d, std::max<size_t>(im.bytes.size(), 16));
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(D.d, im.bytes.data(), im.bytes.size(), cudaMemcpyHostToDevice, st);
}

template <class T>
BatchSection one_block_each(BatchImage& im, const std::vector<T>& items) {
  std::vector<int> ones(items.size(), 1);
  return im.section(items, ones, 32, 0);
}

// ---------------------------------------------------------------------------
// Lockstep GMRES over several instances (each with its own sigma), right
// preconditioned, flexible form, classical Gram-Schmidt applied twice: the
// single-problem cycle's arithmetic (below 16,384 unknowns its results equal
// stab_solve's bit for bit; above, stab_solve orthogonalises with selective
// reorthogonalisation instead).
// ---------------------------------------------------------------------------
struct BgmInst {
  StabHandle* h;
  cd sigma;
  GmresWs W;
  GmDev D;
  int m;
  bool pc;
  double bnorm = 0.0;
  bool converged = false;
  int iters = 0;
  int cycles = 0;
};

struct BatchGmres {
  std::vector<BgmInst> I;
  int device = 0;
  cudaStream_t st = nullptr;
  int maxm = 0;
  DevImage img;
  BatchImage im;
  size_t devs_off = 0, reps_off = 0, done_off = 0, bptr_off = 0, scal_off = 0;
  BatchSection head, scale[kMaxGmresM], tail_gemv, tail_vec, tail_norm, bnorm_sec;
  PcBatchPlan pc[kMaxGmresM];
  JvBatchPlan jv[kMaxGmresM], tail_jv;
  CgsBatchPlan cgs[kMaxGmresM];
  bool any_pc[kMaxGmresM] = {};

  const unsigned char* d() const { return (const unsigned char*)img.d; }
  GmDev* devs() const { return (GmDev*)(d() + devs_off); }
  GmReport* reps() const { return (GmReport*)(d() + reps_off); }
  int* done() const { return (int*)(d() + done_off); }

  // workspaces, preconditioners for sigma, images; all on st
  void setup(StabHandle* h0, const std::vector<StabHandle*>& hs, const std::vector<cd>& sig, cudaStream_t stream) {
    st = stream;
    device = hs[0]->device;
    const int count = (int)hs.size();
    I.resize(count);
    for (int i = 0; i < count; ++i) {
      BgmInst& B = I[i];
      B.h = hs[i];
      B.sigma = sig[i];
      B.m = B.h->opts.gmres_m;
      B.pc = B.h->opts.precond != 0;
      GmReport* unused;
      B.W = gmres_ws(B.h, &B.D, &unused);
      if (B.pc && !(B.h->pvalid && B.h->psigma_re == sig[i].real() && B.h->psigma_im == sig[i].imag()))
        ck(B.h, pc_build(B.h, d2(sig[i])), "preconditioner build");
      maxm = std::max(maxm, B.m);
    }
    // per-instance arrays
    std::vector<GmDev> dv(count);
    for (int i = 0; i < count; ++i) dv[i] = I[i].D;
    devs_off = im.put(dv.data(), dv.size() * sizeof(GmDev));
    std::vector<GmReport> rp(count);
    reps_off = im.put(rp.data(), rp.size() * sizeof(GmReport));
    std::vector<int> dn(count, 0);
    done_off = im.put(dn.data(), dn.size() * sizeof(int));
    std::vector<const double*> bp(count);
    for (int i = 0; i < count; ++i) bp[i] = I[i].W.dnorm;
    bptr_off = im.put(bp.data(), bp.size() * sizeof(double*));
    std::vector<double> sc(count, 0.0);
    scal_off = im.put(sc.data(), sc.size() * sizeof(double));
    // ||b|| of every instance
    {
      std::vector<NormJob> nj;
      for (auto& B : I) nj.push_back(NormJob{B.h, B.W.b, B.h->n, B.W.dnorm, 1, nullptr});
      ck(h0, norm_batch_plan(nj, im, bnorm_sec), "norm plan");
    }
    // cycle head: V_0 = r / beta
    {
      std::vector<VecItem> it;
      std::vector<int> bl;
      for (auto& B : I) {
        VecItem v{};
        v.x = B.W.r; v.y = B.W.V; v.norm = B.W.dnorm; v.gate = B.D.flags + 3; v.n = B.h->n; v.op = kVecScale;
        it.push_back(v);
        bl.push_back(vec_blocks<double2>(B.h->n));
      }
      head = im.section(it, bl, 256, 0);
    }
    for (int j = 0; j < maxm; ++j) {
      std::vector<StabHandle*> hp, hj;
      std::vector<const double2*> pq, jvin;
      std::vector<double2*> pz, jvout;
      std::vector<const int*> pg, jg;
      std::vector<double2> shifts;
      std::vector<CgsJob> cj;
      std::vector<VecItem> sv;
      std::vector<int> sb;
      for (auto& B : I) {
        if (j >= B.m) continue;
        const long long n = B.h->n;
        double2* Vj = B.W.V + (size_t)j * n;
        double2* Vn = B.W.V + (size_t)(j + 1) * n;
        double2* zj = B.pc ? B.W.Z + (size_t)j * n : Vj;
        const int* g0 = B.D.flags;
        if (B.pc) {
          hp.push_back(B.h); pq.push_back(Vj); pz.push_back(zj); pg.push_back(g0);
        }
        hj.push_back(B.h); jvin.push_back(zj); jvout.push_back(Vn); jg.push_back(g0);
        shifts.push_back(d2(B.sigma));
        CgsJob c{B.W.V, j + 1, n, Vn, B.W.dh, B.W.dnorm, B.W.partial};
        c.gate = g0;
        cj.push_back(c);
        VecItem v{};
        v.x = Vn; v.y = Vn; v.norm = B.W.dnorm; v.gate = g0; v.n = n; v.op = kVecScale;
        sv.push_back(v);
        sb.push_back(vec_blocks<double2>(n));
      }
      any_pc[j] = !hp.empty();
      if (any_pc[j]) ck(h0, pc_batch_plan(hp, pq.data(), pz.data(), pg.data(), im, pc[j]), "apply plan");
      ck(h0, jv_batch_plan(hj, jvin.data(), jvout.data(), shifts.data(), jg.data(), im, jv[j]), "J v plan");
      ck(h0, cgs2_batch_plan(cj, im, cgs[j]), "CGS2 plan");
      scale[j] = im.section(sv, sb, 256, 0);
    }
    // cycle tail: x += Z y (V y), r = b - (J - sigma) x, ||r||
    {
      std::vector<GemvItem> gi;
      std::vector<int> gb;
      std::vector<StabHandle*> hj;
      std::vector<const double2*> xin;
      std::vector<double2*> rout;
      std::vector<const int*> g3;
      std::vector<double2> shifts;
      std::vector<VecItem> av;
      std::vector<int> ab;
      std::vector<NormJob> nj;
      for (auto& B : I) {
        const long long n = B.h->n;
        GemvItem g{};
        g.V = B.pc ? B.W.Z : B.W.V; g.y = B.W.y; g.x = B.W.x; g.kdev = B.D.flags + 1; g.gate = B.D.flags + 3;
        g.n = n; g.k = B.m;
        gi.push_back(g);
        gb.push_back(vec_blocks<double2>(n));
        hj.push_back(B.h); xin.push_back(B.W.x); rout.push_back(B.W.r); g3.push_back(B.D.flags + 3);
        shifts.push_back(d2(B.sigma));
        VecItem v{};
        v.x = B.W.b; v.y = B.W.r; v.gate = B.D.flags + 3; v.n = n; v.op = kVecAxpby;
        v.a = make_double2(1.0, 0.0); v.b = make_double2(-1.0, 0.0);
        av.push_back(v);
        ab.push_back(vec_blocks<double2>(n));
        nj.push_back(NormJob{B.h, B.W.r, n, B.W.dnorm, 1, B.D.flags + 3});
      }
      tail_gemv = im.section(gi, gb, 256, 0);
      ck(h0, jv_batch_plan(hj, xin.data(), rout.data(), shifts.data(), g3.data(), im, tail_jv), "J v plan");
      tail_vec = im.section(av, ab, 256, 0);
      ck(h0, norm_batch_plan(nj, im, tail_norm), "norm plan");
    }
    if (im.overflow) fail(h0, STAB_ERR_INVALID_ARG, "batched GMRES: too many blocks for one launch");
    for (auto& B : I) ck(B.h, cudaStreamSynchronize(B.h->stream), "sync");  // workspaces and factors ready
    ck(h0, upload(img, device, st, im), "parameter image");
    for (int j = 0; j < maxm; ++j) ck(h0, jv_batch_zero_eps(jv[j], st), "epsilon");
    ck(h0, jv_batch_zero_eps(tail_jv, st), "epsilon");
    for (auto& B : I)
      if (B.h->opts.eps_mode == 2) B.h->last_eps_mode = 2;
  }

  // (J_i - sigma_i I) x_i = b_i for the instances with take[i]; returns after all have converged or hit
  // their restart limits.  b_i is read from B.W.b (filled by the caller) and the solution left in B.W.x.
  void run(StabHandle* h0, const std::vector<char>& take) {
    const int count = (int)I.size();
    std::vector<double> bn(count, 0.0);
    const unsigned char* D = d();
    ck(h0, norm_batch_launch(bnorm_sec, D, st), "norm");
    k_gather<<<1, 256, 0, st>>>((const double* const*)(D + bptr_off), (double*)(D + scal_off), count);
    ck(h0, cudaMemcpyAsync(bn.data(), D + scal_off, count * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
    ck(h0, cudaStreamSynchronize(st), "sync");
    std::vector<int> done(count, 1);
    int left = 0;
    for (int i = 0; i < count; ++i) {
      BgmInst& B = I[i];
      B.converged = false;
      B.iters = 0;
      B.cycles = 0;
      if (!take[i]) continue;
      B.bnorm = bn[i];
      if (!(bn[i] < INFINITY)) fail(B.h, STAB_ERR_NUMERIC, "GMRES: right-hand side is not finite");
      ck(B.h, cudaMemsetAsync(B.W.x, 0, B.h->n * sizeof(double2), st), "memset");
      if (bn[i] == 0.0) { B.converged = true; continue; }
      ck(B.h, kry_copy(B.h, B.W.b, B.W.r, B.h->n), "copy");
      k_gm_tol<<<1, 1, 0, st>>>(B.D, B.h->opts.gmres_tol);
      done[i] = 0;
      ++left;
    }
    ck(h0, cudaMemcpyAsync((void*)done_ptr(), done.data(), count * sizeof(int), cudaMemcpyHostToDevice, st), "copy");
    k_bgm_begin<<<count, 32, 0, st>>>(devs(), done_ptr(), 0.0);
    std::vector<GmReport> rep(count);
    for (int cycle = 0; left > 0; ++cycle) {
      k_bgm_init<<<count, 64, 0, st>>>(devs());
      k_bvec<<<head.blocks, 256, 0, st>>>((const VecItem*)(D + head.items), (const int*)(D + head.start), head.count);
      for (int j = 0; j < maxm; ++j) {
        if (any_pc[j]) ck(h0, pc_batch_launch(pc[j], D, st), "block apply");
        ck(h0, jv_batch_launch(jv[j], D, st), "J v");
        ck(h0, cgs2_batch_launch(cgs[j], D, st), "CGS2");
        k_bgm_step<<<count, 32, 0, st>>>(devs(), j);
        k_bvec<<<scale[j].blocks, 256, 0, st>>>((const VecItem*)(D + scale[j].items), (const int*)(D + scale[j].start),
                                                scale[j].count);
      }
      k_bgm_solve<<<count, 64, 0, st>>>(devs());
      k_bgemv<<<tail_gemv.blocks, 256, 0, st>>>((const GemvItem*)(D + tail_gemv.items),
                                                (const int*)(D + tail_gemv.start), tail_gemv.count);
      ck(h0, jv_batch_launch(tail_jv, D, st), "J v");
      k_bvec<<<tail_vec.blocks, 256, 0, st>>>((const VecItem*)(D + tail_vec.items), (const int*)(D + tail_vec.start),
                                              tail_vec.count);
      ck(h0, norm_batch_launch(tail_norm, D, st), "norm");
      k_bgm_report<<<count, 32, 0, st>>>(devs(), reps());
      ck(h0, cudaGetLastError(), "batched GMRES cycle");
      ck(h0, cudaMemcpyAsync(rep.data(), reps(), count * sizeof(GmReport), cudaMemcpyDeviceToHost, st), "report");
      ck(h0, cudaStreamSynchronize(st), "sync");
      std::vector<int> stop;
      for (int i = 0; i < count; ++i) {
        if (done[i]) continue;
        BgmInst& B = I[i];
        B.iters += rep[i].jend;
        B.cycles++;
        B.h->stats.jv_calls += rep[i].jend + 1;
        if (rep[i].status) fail(B.h, STAB_ERR_NUMERIC, "GMRES: non-finite Krylov vector");
        if (!(rep[i].beta < INFINITY)) fail(B.h, STAB_ERR_NUMERIC, "GMRES: non-finite residual");
        if (rep[i].beta <= B.h->opts.gmres_tol * B.bnorm) {
          B.converged = true;
          done[i] = 1;
          --left;
        } else if (B.cycles >= B.h->opts.gmres_max_restarts) {
          done[i] = 1;
          --left;
          stop.push_back(i);
        }
      }
      if (!stop.empty()) {  // restart limit: leave the instance out of further cycles
        ck(h0, cudaMemcpyAsync((void*)done_ptr(), done.data(), count * sizeof(int), cudaMemcpyHostToDevice, st),
           "copy");
        k_bgm_begin<<<count, 32, 0, st>>>(devs(), done_ptr(), 0.0);
      }
    }
    for (int i = 0; i < count; ++i)
      if (take[i]) {
        I[i].h->stats.gmres_iterations += I[i].iters;
        I[i].h->stats.gmres_solves += 1;
        if (I[i].h->opts.eps_mode != 2) I[i].h->last_eps_mode = I[i].h->opts.eps_mode;
      }
  }
  int* done_ptr() const { return (int*)(d() + done_off); }
};

}  // namespace

namespace {

// Make the batch's stream the instances' stream for the duration of a
// lockstep solve (ordered after their own streams, which are ordered after
// it again on return), so that the per-instance helpers run on it too.
struct StreamSwap {
  stab_jv_batch_s* B;
  std::vector<cudaStream_t> saved;
  explicit StreamSwap(stab_jv_batch_s* b) : B(b) {
    batch_order_begin(B);
    for (StabHandle* h : B->hs) {
      saved.push_back(h->stream);
      h->stream = B->stream;
    }
  }
  ~StreamSwap() {
    for (size_t i = 0; i < B->hs.size(); ++i) B->hs[i]->stream = saved[i];
    batch_order_end(B);
  }
};

bool batchable_solver(const StabHandle* h) {
  return h->opts.gmres_basis_prec == 64 && h->opts.lgmres_k == 0 && h->opts.gmres_inner_m == 0 &&
         h->opts.precond != 2;
}

}  // namespace

extern "C" stab_status stab_jv_batch_solve(stab_jv_batch B, const double* sigmas, const void* const* rhs,
                                           void* const* x, int* iters) {
  if (!B) return STAB_ERR_INVALID_ARG;
  const int count = (int)B->hs.size();
  if (!sigmas || !rhs || !x) {
    B->err = "stab_jv_batch_solve: null argument list";
    return STAB_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    if (!rhs[i] || !x[i]) {
      B->err = "stab_jv_batch_solve: null vector of instance " + std::to_string(i);
      return STAB_ERR_INVALID_ARG;
    }
    if (!batchable_solver(B->hs[i])) {
      B->err = "stab_jv_batch_solve: instance " + std::to_string(i) + " uses an FP32 basis, LGMRES, a nested inner solver or the reduced-operator preconditioner";
      return STAB_ERR_UNSUPPORTED;
    }
  }
  StabHandle* h0 = B->hs[0];
  stab_status result = STAB_OK;
  StreamSwap swap(B);
  try {
    std::vector<cd> sig(count);
    for (int i = 0; i < count; ++i) sig[i] = cd(sigmas[2 * i], sigmas[2 * i + 1]);
    BatchGmres G;
    G.setup(h0, B->hs, sig, B->stream);
    for (int i = 0; i < count; ++i)
      ck(G.I[i].h, kry_copy(G.I[i].h, (const double2*)rhs[i], G.I[i].W.b, G.I[i].h->n), "copy b");
    G.run(h0, std::vector<char>(count, 1));
    for (int i = 0; i < count; ++i) {
      ck(G.I[i].h, kry_copy(G.I[i].h, G.I[i].W.x, (double2*)x[i], G.I[i].h->n), "copy x");
      if (iters) iters[i] = G.I[i].iters;
      if (!G.I[i].converged && result == STAB_OK) {
        result = STAB_ERR_NOT_CONVERGED;
        B->err = "stab_jv_batch_solve: instance " + std::to_string(i) + " reached its GMRES restart limit";
      }
    }
    ck(h0, cudaStreamSynchronize(B->stream), "sync");
  } catch (Fail& f) {
    for (StabHandle* h : B->hs)
      if (!h->err.empty()) B->err = "stab_jv_batch_solve: " + h->err;
    result = f.st;
  }
  return result;
}

// Cayley-IRAM of every instance in lockstep: the Arnoldi steps j of all
// instances that have not finished run as one launch per phase (J v with
// their taus, the lockstep GMRES with their sigmas, CGS2, the Hessenberg
// entries), the implicit restarts as one launch (one CTA per instance).
// Instances with smaller ncv sit out the steps beyond their ncv; after a
// restart every instance resumes at its own nev.
extern "C" stab_status stab_jv_batch_eigs(stab_jv_batch B, stab_eig_job* jobs) {
  if (!B) return STAB_ERR_INVALID_ARG;
  const int count = (int)B->hs.size();
  if (!jobs) {
    B->err = "stab_jv_batch_eigs: null job list";
    return STAB_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    StabHandle* h = B->hs[i];
    const stab_eig_job& J = jobs[i];
    if (J.nev < 1 || J.ncv <= J.nev || J.ncv > 512 || J.ncv > h->n || !(J.tol > 0) || !J.lambda) {
      B->err = "stab_jv_batch_eigs: job " + std::to_string(i) + " needs 1 <= nev < ncv <= min(n, 512), tol > 0, lambda";
      return STAB_ERR_INVALID_ARG;
    }
    if (!batchable_solver(h)) {
      B->err = "stab_jv_batch_eigs: instance " + std::to_string(i) + " uses an FP32 basis, LGMRES, a nested inner solver or the reduced-operator preconditioner";
      return STAB_ERR_UNSUPPORTED;
    }
  }
  struct Inst {
    StabHandle* h;
    stab_eig_job* job;
    cd sigma, tau;
    int k, m;
    double2 *V, *f, *xw, *tmp, *partial, *dh;
    double* dn;
    RestartWs RW;
    int j0 = 0;
    bool active = true, first = true;
    int conv = 0, restarts = 0;
    std::vector<cd> theta;
    stab_status st = STAB_OK;
    stab_stats s0;
    std::chrono::steady_clock::time_point t0;
  };
  StabHandle* h0 = B->hs[0];
  cudaStream_t st = B->stream;
  stab_status result = STAB_OK;
  StreamSwap swap(B);
  std::vector<Inst> I(count);
  try {
    int maxm = 0;
    std::vector<cd> sig(count);
    for (int i = 0; i < count; ++i) {
      Inst& S = I[i];
      S.h = B->hs[i];
      S.job = &jobs[i];
      S.sigma = cd(jobs[i].sigma_re, jobs[i].sigma_im);
      S.tau = cd(jobs[i].tau_re, jobs[i].tau_im);
      S.k = jobs[i].nev;
      S.m = jobs[i].ncv;
      S.s0 = S.h->stats;
      S.t0 = std::chrono::steady_clock::now();
      S.theta.assign(S.k, cd(0.0));
      sig[i] = S.sigma;
      maxm = std::max(maxm, S.m);
      StabHandle* h = S.h;
      const long long n = h->n;
      if (h->opts.precond != 0 && !(h->pvalid && h->psigma_re == S.sigma.real() && h->psigma_im == S.sigma.imag())) {
        auto tp = std::chrono::steady_clock::now();
        ck(h, pc_build(h, d2(S.sigma)), "preconditioner build");
        ck(h, cudaStreamSynchronize(st), "sync");
        h->stats.seconds_precond += std::chrono::duration<double>(std::chrono::steady_clock::now() - tp).count();
      }
      const size_t part = (size_t)kry_partial_elems(n, S.m);
      const size_t rws = restart_ws_elems(S.m, S.k);
      const size_t need = (size_t)S.m * n + 2 * (size_t)n + (size_t)(S.k + 1) * n + part + 2 * S.m + 4 + rws;
      double2* base = ensure(h, &h->d_ir, &h->ir_elems, need);
      S.V = base;
      S.f = S.V + (size_t)S.m * n;
      S.xw = S.f + n;
      S.tmp = S.xw + n;
      S.partial = S.tmp + (size_t)(S.k + 1) * n;
      S.dh = S.partial + part;
      S.dn = (double*)(S.dh + 2 * S.m);
      S.RW = restart_ws(S.dh + 2 * S.m + 4, S.m, S.k);
      if (jobs[i].v0) ck(h, kry_copy(h, (const double2*)jobs[i].v0, S.f, n), "copy v0");
      else {
        std::vector<double> sv;
        splitmix_start(h->opts.seed, n, sv);
        ck(h, cudaMemcpyAsync(S.f, sv.data(), sizeof(double) * sv.size(), cudaMemcpyHostToDevice, st), "copy start");
        ck(h, cudaStreamSynchronize(st), "sync");
      }
      k_zero<<<1, 256, 0, st>>>(S.RW.H, S.m * S.m);
    }
    // the lockstep GMRES: b = (J - tau) v_j in xw, x = the new f
    BatchGmres G;
    G.setup(h0, B->hs, sig, st);
    // Arnoldi-step phases per j, gated per (instance, j): gate[i * maxm + j] != 0 while instance i sits out step j
    BatchImage im;
    std::vector<int> gate_host((size_t)count * maxm, 1);
    const size_t gate_off = im.put(gate_host.data(), gate_host.size() * sizeof(int));
    std::vector<const double*> dnp(count);
    for (int i = 0; i < count; ++i) dnp[i] = I[i].dn;
    const size_t dnp_off = im.put(dnp.data(), dnp.size() * sizeof(double*));
    std::vector<double> zeros(count, 0.0);
    const size_t beta_off = im.put(zeros.data(), zeros.size() * sizeof(double));
    // gate pointers are only known after the upload: items refer to them by offset, patched below
    std::vector<BatchSection> s_norm(maxm), s_hsub(maxm), s_scale(maxm), s_hcol(maxm);
    std::vector<JvBatchPlan> p_jv(maxm);
    std::vector<CgsBatchPlan> p_cgs(maxm);
    DevImage img;
    // two passes: the items hold the gates' device addresses, so the image is sized by a dry build,
    // allocated, then built again against its device base
    auto build = [&](const unsigned char* dbase) {
      BatchImage b2;
      b2.put(gate_host.data(), gate_host.size() * sizeof(int));
      b2.put(dnp.data(), dnp.size() * sizeof(double*));
      b2.put(zeros.data(), zeros.size() * sizeof(double));
      const int* gbase = (const int*)(dbase + gate_off);
      for (int j = 0; j < maxm; ++j) {
        std::vector<NormJob> nj;
        std::vector<HItem> hs_, hc;
        std::vector<VecItem> sv;
        std::vector<int> sb;
        std::vector<StabHandle*> hj;
        std::vector<const double2*> vin;
        std::vector<double2*> vout;
        std::vector<const int*> gj;
        std::vector<double2> shifts;
        std::vector<CgsJob> cj;
        for (int i = 0; i < count; ++i) {
          Inst& S = I[i];
          if (j >= S.m) continue;
          const long long n = S.h->n;
          const int* g = gbase + (size_t)i * maxm + j;
          double2* Vj = S.V + (size_t)j * n;
          nj.push_back(NormJob{S.h, S.f, n, S.dn, 1, g});
          if (j > 0) hs_.push_back(HItem{S.RW.H, nullptr, S.dn, g, S.m, j, 0, 0});
          VecItem v{};
          v.x = S.f; v.y = Vj; v.norm = S.dn; v.gate = g; v.n = n; v.op = kVecScale;
          sv.push_back(v);
          sb.push_back(vec_blocks<double2>(n));
          hj.push_back(S.h); vin.push_back(Vj); vout.push_back(S.xw); gj.push_back(g); shifts.push_back(d2(S.tau));
          CgsJob c{S.V, j + 1, n, S.f, S.dh, S.dn, S.partial};
          c.gate = g;
          cj.push_back(c);
          hc.push_back(HItem{S.RW.H, S.dh, S.dn, g, S.m, j, 1, 0});
        }
        ck(h0, norm_batch_plan(nj, b2, s_norm[j]), "norm plan");
        s_hsub[j] = one_block_each(b2, hs_);
        s_scale[j] = b2.section(sv, sb, 256, 0);
        ck(h0, jv_batch_plan(hj, vin.data(), vout.data(), shifts.data(), gj.data(), b2, p_jv[j]), "J v plan");
        ck(h0, cgs2_batch_plan(cj, b2, p_cgs[j]), "CGS2 plan");
        s_hcol[j] = one_block_each(b2, hc);
      }
      return b2;
    };
    {
      BatchImage dry = build(nullptr);
      ck(h0, dev_alloc_stream(B->device, st, &img.d, std::max<size_t>(dry.bytes.size(), 16)), "parameter image");
      img.st = st;
      im = build((const unsigned char*)img.d);
      if (im.overflow) fail(h0, STAB_ERR_INVALID_ARG, "stab_jv_batch_eigs: too many blocks for one launch");
      ck(h0, cudaMemcpyAsync(img.d, im.bytes.data(), im.bytes.size(), cudaMemcpyHostToDevice, st), "image");
    }
    const unsigned char* D = (const unsigned char*)img.d;
    int* d_gate = (int*)(D + gate_off);
    for (int j = 0; j < maxm; ++j) ck(h0, jv_batch_zero_eps(p_jv[j], st), "epsilon");
    auto push_gates = [&](int restart_pass) {
      for (int i = 0; i < count; ++i)
        for (int j = 0; j < maxm; ++j)
          gate_host[(size_t)i * maxm + j] = (!I[i].active || j < I[i].j0 || j >= I[i].m) ? 1 : 0;
      (void)restart_pass;
      ck(h0, cudaMemcpyAsync(d_gate, gate_host.data(), gate_host.size() * sizeof(int), cudaMemcpyHostToDevice, st),
         "gates");
    };
    std::vector<double> beta(count);
    for (int restart = 0;; ++restart) {
      push_gates(restart);
      int jmin = maxm;
      for (auto& S : I)
        if (S.active) jmin = std::min(jmin, S.j0);
      for (int j = jmin; j < maxm; ++j) {
        std::vector<char> take(count, 0);
        bool any = false;
        for (int i = 0; i < count; ++i) take[i] = I[i].active && j >= I[i].j0 && j < I[i].m, any |= take[i];
        if (!any) continue;
        ck(h0, norm_batch_launch(s_norm[j], D, st), "norm");
        k_gather<<<1, 256, 0, st>>>((const double* const*)(D + dnp_off), (double*)(D + beta_off), count);
        ck(h0, cudaMemcpyAsync(beta.data(), D + beta_off, count * sizeof(double), cudaMemcpyDeviceToHost, st), "copy");
        ck(h0, cudaStreamSynchronize(st), "sync");
        bool dropped = false;
        for (int i = 0; i < count; ++i) {
          if (!take[i]) continue;
          if (!(beta[i] < INFINITY) || beta[i] == 0.0) {
            I[i].st = beta[i] == 0.0 ? STAB_ERR_BREAKDOWN : STAB_ERR_NUMERIC;
            I[i].h->err = beta[i] == 0.0 ? "IRAM: Arnoldi breakdown (invariant subspace)"
                                         : "IRAM: non-finite residual vector";
            I[i].active = false;
            take[i] = 0;
            dropped = true;
          }
        }
        if (dropped) push_gates(restart);
        if (s_hsub[j].count) k_bhess<<<s_hsub[j].count, 32, 0, st>>>((const HItem*)(D + s_hsub[j].items), s_hsub[j].count);
        k_bvec<<<s_scale[j].blocks, 256, 0, st>>>((const VecItem*)(D + s_scale[j].items),
                                                  (const int*)(D + s_scale[j].start), s_scale[j].count);
        ck(h0, jv_batch_launch(p_jv[j], D, st), "J v");
        for (int i = 0; i < count; ++i)
          if (take[i]) {
            I[i].h->stats.jv_calls++;
            ck(I[i].h, kry_copy(I[i].h, I[i].xw, G.I[i].W.b, I[i].h->n), "copy b");
          }
        G.run(h0, take);
        for (int i = 0; i < count; ++i)
          if (take[i]) {
            if (!G.I[i].converged && I[i].st == STAB_OK) I[i].st = STAB_ERR_NOT_CONVERGED;
            ck(I[i].h, kry_copy(I[i].h, G.I[i].W.x, I[i].f, I[i].h->n), "copy x");
          }
        ck(h0, cgs2_batch_launch(p_cgs[j], D, st), "CGS2");
        k_bhess<<<s_hcol[j].count, 64, 0, st>>>((const HItem*)(D + s_hcol[j].items), s_hcol[j].count);
        ck(h0, cudaGetLastError(), "Arnoldi step");
        for (int i = 0; i < count; ++i)
          if (take[i]) I[i].h->stats.arnoldi_steps++;
      }
      // implicit restarts of every active instance, one CTA each
      std::vector<RsItem> rs;
      std::vector<int> idx;
      for (int i = 0; i < count; ++i) {
        Inst& S = I[i];
        S.first = false;
        if (!S.active) continue;
        RsItem r{};
        r.w = S.RW; r.sg = d2(S.sigma); r.ta = d2(S.tau); r.tol = S.job->tol; r.fnorm = S.dn; r.gate = nullptr;
        r.m = S.m; r.k = S.k; r.finish = S.restarts >= S.h->opts.max_restarts;
        rs.push_back(r);
        idx.push_back(i);
      }
      if (rs.empty()) break;
      {
        BatchImage ri;
        const BatchSection rsec = one_block_each(ri, rs);
        DevImage rimg;
        ck(h0, upload(rimg, B->device, st, ri), "restart items");
        k_brestart<<<rsec.count, 32, 0, st>>>((const RsItem*)((const unsigned char*)rimg.d + rsec.items), rsec.count);
        ck(h0, cudaGetLastError(), "restart kernel");
        std::vector<std::vector<double>> out(rs.size());
        for (size_t q = 0; q < rs.size(); ++q) {
          Inst& S = I[idx[q]];
          out[q].assign(2 * S.k + S.k + 4, 0.0);
          ck(h0, cudaMemcpyAsync(out[q].data(), S.RW.out_theta, sizeof(double2) * S.k, cudaMemcpyDeviceToHost, st),
             "copy");
          ck(h0, cudaMemcpyAsync(out[q].data() + 2 * S.k, S.RW.est, sizeof(double) * (S.k + 4),
                                 cudaMemcpyDeviceToHost, st), "copy");
        }
        ck(h0, cudaStreamSynchronize(st), "sync");
        for (size_t q = 0; q < rs.size(); ++q) {
          Inst& S = I[idx[q]];
          const double* scal = out[q].data() + 3 * S.k;
          if (scal[0] < 0) {
            S.st = STAB_ERR_NUMERIC;
            S.h->err = "IRAM: Hessenberg QR failed";
            S.active = false;
            continue;
          }
          S.conv = (int)scal[0];
          for (int t = 0; t < S.k; ++t) S.theta[t] = cd(out[q][2 * t], out[q][2 * t + 1]);
          const bool finish = S.restarts >= S.h->opts.max_restarts;
          if (S.conv == S.k || finish) {
            if (S.conv < S.k && S.st == STAB_OK) {
              S.st = STAB_ERR_NOT_CONVERGED;
              S.h->err = "stab_eigs: IRAM restart limit reached";
            }
            S.active = false;
            S.j0 = -1;  // finished: extract below
            continue;
          }
          S.h->stats.restarts++;
          S.restarts++;
          const long long n = S.h->n;
          ck(S.h, kry_update_basis(S.h, S.V, S.m, S.k + 1, n, (const double2*)S.RW.Qc, S.tmp), "V Q");
          k_f_update<<<1024, 256, 0, st>>>(S.tmp + (size_t)S.k * n, S.f, n, S.RW.coef);
          ck(S.h, cudaMemcpyAsync(S.V, S.tmp, sizeof(double2) * (size_t)S.k * n, cudaMemcpyDeviceToDevice, st),
             "copy V");
          S.j0 = S.k;
        }
        ck(h0, cudaStreamSynchronize(st), "sync");  // the restart items' image is released after this
      }
      bool any = false;
      for (auto& S : I) any |= S.active;
      if (!any) break;
    }
    // eigenpairs of every instance that finished its restarts: as stab_eigs
    for (int i = 0; i < count; ++i) {
      Inst& S = I[i];
      stab_eig_job& J = *S.job;
      J.nconv = 0;
      if (S.j0 != -1) continue;  // failed before finishing
      StabHandle* h = S.h;
      const long long n = h->n;
      double2* X = S.tmp;
      ck(h, kry_update_basis(h, S.V, S.m, S.k, n, (const double2*)S.RW.Qc, X), "V Y");
      for (int q = 0; q < S.k; ++q) {
        const cd t = S.theta[q];
        const cd lam = (S.sigma * t - S.tau) / (t - 1.0);
        J.lambda[2 * q] = lam.real();
        J.lambda[2 * q + 1] = lam.imag();
        double2* xq = X + (size_t)q * n;
        ck(h, launch_norm2(h, xq, n, S.dn, 1), "norm");
        ck(h, kry_scale(h, xq, n, S.dn, nullptr), "normalise");
        if (J.resid) {
          ck(h, jv_apply(h, xq, S.xw, d2(lam), 2), "J x");
          ck(h, launch_norm2(h, S.xw, n, S.dn, 1), "norm");
          J.resid[q] = read_scalar(h, S.dn);
        }
        if (J.vecs) ck(h, kry_copy(h, xq, (double2*)J.vecs + (size_t)q * n, n), "copy vector");
      }
      J.nconv = S.conv;
    }
    ck(h0, cudaStreamSynchronize(st), "sync");
  } catch (Fail& f) {
    result = f.st;
    for (StabHandle* h : B->hs)
      if (!h->err.empty()) B->err = "stab_jv_batch_eigs: " + h->err;
  }
  for (int i = 0; i < count; ++i) {
    Inst& S = I[i];
    if (!S.h) continue;
    stab_eig_job& J = jobs[i];
    J.status = result != STAB_OK ? result : S.st;
    S.h->stats.seconds_total += std::chrono::duration<double>(std::chrono::steady_clock::now() - S.t0).count();
    stab_stats d = S.h->stats;
    d.jv_calls -= S.s0.jv_calls;
    d.gmres_iterations -= S.s0.gmres_iterations;
    d.gmres_solves -= S.s0.gmres_solves;
    d.arnoldi_steps -= S.s0.arnoldi_steps;
    d.restarts -= S.s0.restarts;
    d.precond_builds -= S.s0.precond_builds;
    d.seconds_total -= S.s0.seconds_total;
    d.seconds_precond -= S.s0.seconds_precond;
    J.stats = d;
    if (result == STAB_OK && S.st != STAB_OK && S.st != STAB_ERR_NOT_CONVERGED) result = S.st;
  }
  if (result == STAB_OK)
    for (int i = 0; i < count; ++i)
      if (jobs[i].status == STAB_ERR_NOT_CONVERGED) { result = STAB_ERR_NOT_CONVERGED; break; }
  return result;
}
