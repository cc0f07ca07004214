// Inner linear solver and outer eigensolver, orchestrated from the host with
// all vector work on the device:
//  * restarted GMRES(m) (Sec. "Iterative solvers") in flexible,
//    right-preconditioned form, x0 = 0, stopping on ||b - A x|| <= tol ||b||;
//  * the Cayley-transformed implicitly restarted Arnoldi method
//    (Algorithm iram, Eqs. cayley_transform / cayley_arnoldi / ritz_estimate)
//    with CGS2 orthogonalisation and exact shifts.
// The small (m x m) Hessenberg algebra of the restart stays on the device
// (k_restart); GMRES's Givens least-squares update runs on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "hess_dev.cuh"
#include "hessenberg.h"
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
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  ck(h, cudaMalloc(p, need * sizeof(double2)), "workspace allocation");
  *have = need;
  return *p;
}

// GMRES workspace layout (complex elements)
struct GmresWs {
  double2 *V, *Z, *r, *partial, *dh, *y;
  double* dnorm;
};

GmresWs gmres_ws(StabHandle* h) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond == 1;
  const size_t part = (size_t)kry_partial_elems(n, m + 1);
  size_t need = (size_t)(m + 1) * n + (pc ? (size_t)m * n : 0) + n + part + 2 * (m + 1) + (m + 1) + 4;
  double2* base = ensure(h, &h->d_gm, &h->gm_elems, need);
  GmresWs w;
  w.V = base;
  w.Z = pc ? base + (size_t)(m + 1) * n : nullptr;
  w.r = base + (size_t)(m + 1) * n + (pc ? (size_t)m * n : 0);
  w.partial = w.r + n;
  w.dh = w.partial + part;
  w.y = w.dh + 2 * (m + 1);
  w.dnorm = (double*)(w.y + (m + 1));
  return w;
}

double read_scalar(StabHandle* h, const double* d) {
  double v;
  ck(h, cudaMemcpyAsync(&v, d, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "read scalar");
  ck(h, cudaStreamSynchronize(h->stream), "sync");
  return v;
}

// (J - sigma I) x = b.  Returns the iteration count; sets *converged.
int gmres(StabHandle* h, cd sigma, const double2* b, double2* x, int eps_mode, bool* converged) {
  const long long n = h->n;
  const int m = h->opts.gmres_m;
  const bool pc = h->opts.precond == 1;
  const double tol = h->opts.gmres_tol;
  GmresWs W = gmres_ws(h);
  ck(h, launch_norm2(h, b, n, W.dnorm, 1), "norm");
  const double bnorm = read_scalar(h, W.dnorm);
  ck(h, cudaMemsetAsync(x, 0, n * sizeof(double2), h->stream), "memset");
  *converged = false;
  if (!(bnorm < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: right-hand side is not finite");
  if (bnorm == 0.0) { *converged = true; return 0; }
  ck(h, kry_copy(h, b, W.r, n), "copy");
  double beta = bnorm;
  int total = 0;
  std::vector<cd> H((size_t)(m + 1) * m), g(m + 1), sn(m), hcol(2 * (m + 1));
  std::vector<double> cs(m);
  std::vector<double> hbuf(2 * (m + 1) + 2);
  for (int cycle = 0; cycle < h->opts.gmres_max_restarts; ++cycle) {
    // V_0 = r / beta (W.dnorm holds beta on the device)
    ck(h, kry_scale(h, W.r, n, W.dnorm, W.V), "scale");
    std::fill(g.begin(), g.end(), cd(0.0));
    g[0] = beta;
    int jend = 0;
    for (int j = 0; j < m; ++j) {
      double2* Vj = W.V + (size_t)j * n;
      double2* Vn = W.V + (size_t)(j + 1) * n;
      double2* zj = Vj;
      if (pc) {
        zj = W.Z + (size_t)j * n;
        ck(h, pc_apply(h, Vj, zj), "preconditioner apply");
      }
      ck(h, jv_apply(h, zj, Vn, d2(sigma), eps_mode), "J v");
      ck(h, kry_cgs2(h, W.V, j + 1, n, Vn, W.dh, W.dnorm, W.partial), "CGS2");
      // fetch h(0..j) and ||w|| in one copy (dnorm follows dh + 2(m+1) + (m+1))
      ck(h, cudaMemcpyAsync(hbuf.data(), W.dh, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, h->stream), "copy h");
      double wn;
      ck(h, cudaMemcpyAsync(&wn, W.dnorm, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy norm");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
      for (int i = 0; i <= j; ++i) hcol[i] = cd(hbuf[2 * i], hbuf[2 * i + 1]);
      hcol[j + 1] = wn;
      if (!(wn < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: non-finite Krylov vector");
      for (int i = 0; i < j; ++i) {  // previous rotations
        cd a = hcol[i], bb = hcol[i + 1];
        hcol[i] = cs[i] * a + sn[i] * bb;
        hcol[i + 1] = -std::conj(sn[i]) * a + cs[i] * bb;
      }
      hess::givens_ls(hcol[j], hcol[j + 1], cs[j], sn[j]);
      hcol[j] = cs[j] * hcol[j] + sn[j] * hcol[j + 1];
      hcol[j + 1] = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      ++total;
      jend = j + 1;
      const double res = std::abs(g[j + 1]);
      if (res <= tol * bnorm || wn == 0.0) break;
      ck(h, kry_scale(h, Vn, n, W.dnorm, nullptr), "scale");
    }
    // y = R^{-1} g (upper triangular jend x jend)
    std::vector<cd> y(jend);
    for (int i = jend - 1; i >= 0; --i) {
      cd s = g[i];
      for (int l = i + 1; l < jend; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    ck(h, cudaMemcpyAsync(W.y, y.data(), sizeof(double2) * jend, cudaMemcpyHostToDevice, h->stream), "copy y");
    ck(h, kry_gemv_add(h, pc ? W.Z : W.V, jend, n, W.y, x), "x update");
    // true residual r = b - (J - sigma I) x
    ck(h, jv_apply(h, x, W.r, d2(sigma), eps_mode), "J v");
    ck(h, kry_axpby(h, make_double2(1.0, 0.0), b, make_double2(-1.0, 0.0), W.r, n), "axpby");
    ck(h, launch_norm2(h, W.r, n, W.dnorm, 1), "norm");
    beta = read_scalar(h, W.dnorm);
    if (!(beta < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: non-finite residual");
    if (beta <= tol * bnorm) { *converged = true; break; }
  }
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
