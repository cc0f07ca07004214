// Inner linear solver and outer eigensolver, orchestrated from the host with
// all vector work on the device:
//  * restarted GMRES(m) (Sec. "Iterative solvers") in flexible,
//    right-preconditioned form, x0 = 0, stopping on ||b - A x|| <= tol ||b||;
//  * the Cayley-transformed implicitly restarted Arnoldi method
//    (Algorithm iram, Eqs. cayley_transform / cayley_arnoldi / ritz_estimate)
//    with CGS2 orthogonalisation and exact shifts.
// Only the small (m x m) Hessenberg algebra runs on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

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
    bool done = false;
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
      if (res <= tol * bnorm || wn == 0.0) { done = true; break; }
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
    (void)done;
    if (!(beta < INFINITY)) fail(h, STAB_ERR_NUMERIC, "GMRES: non-finite residual");
    if (beta <= tol * bnorm) { *converged = true; break; }
  }
  h->stats.gmres_iterations += total;
  h->stats.gmres_solves += 1;
  return total;
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
    // IRAM workspace: V (m n), f (n), x (n), tmp ((k+1) n), Q (m (k+1)), partials, dh, scalars
    const size_t part = (size_t)kry_partial_elems(n, m);
    const size_t need = (size_t)m * n + 2 * (size_t)n + (size_t)(k + 1) * n + (size_t)m * (k + 1) + part + 2 * m + 4;
    double2* base = ensure(h, &h->d_ir, &h->ir_elems, need);
    double2* V = base;
    double2* f = V + (size_t)m * n;
    double2* xw = f + n;
    double2* tmp = xw + n;
    double2* dQ = tmp + (size_t)(k + 1) * n;
    double2* partial = dQ + (size_t)m * (k + 1);
    double2* dh = partial + part;
    double* dn = (double*)(dh + 2 * m);
    // start vector
    if (v0) ck(h, kry_copy(h, (const double2*)v0, f, n), "copy v0");
    else {
      std::vector<double> sv;
      splitmix_start(h->opts.seed, n, sv);
      ck(h, cudaMemcpyAsync(f, sv.data(), sizeof(double) * sv.size(), cudaMemcpyHostToDevice, h->stream), "copy start");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
    }
    std::vector<cd> H((size_t)m * m, 0.0), theta(m), Y((size_t)m * m), Q((size_t)m * m);
    std::vector<double> hbuf(2 * m);
    std::vector<int> order(m);
    std::vector<double> est(k);
    int j0 = 0;
    bool first = true;
    int conv_count = 0;
    double fnorm = 0.0;
    for (int restart = 0;; ++restart) {
      for (int j = j0; j < m; ++j) {
        ck(h, launch_norm2(h, f, n, dn, 1), "norm");
        const double beta = read_scalar(h, dn);
        if (!(beta < INFINITY)) fail(h, STAB_ERR_NUMERIC, "IRAM: non-finite residual vector");
        if (beta == 0.0) fail(h, STAB_ERR_BREAKDOWN, "IRAM: Arnoldi breakdown (invariant subspace)");
        if (!first || j > 0) H[(size_t)j * m + j - 1] = beta;
        double2* Vj = V + (size_t)j * n;
        ck(h, kry_scale(h, f, n, dn, Vj), "scale");
        // w = C v_j: b = (J - tau I) v_j, then (J - sigma I) x = b
        ck(h, jv_apply(h, Vj, xw, d2(tau), h->opts.eps_mode), "J v");
        bool gconv;
        gmres(h, sigma, xw, f, h->opts.eps_mode, &gconv);
        if (!gconv) result = STAB_ERR_NOT_CONVERGED;
        ck(h, kry_cgs2(h, V, j + 1, n, f, dh, dn, partial), "CGS2");
        ck(h, cudaMemcpyAsync(hbuf.data(), dh, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, h->stream), "copy h");
        ck(h, cudaStreamSynchronize(h->stream), "sync");
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = cd(hbuf[2 * i], hbuf[2 * i + 1]);
        h->stats.arnoldi_steps++;
      }
      first = false;
      fnorm = read_scalar(h, dn);
      // Ritz values, wanted set (largest |theta|; ties: larger Re, then Im lambda)
      if (hess::eig(m, H.data(), theta.data(), Y.data()) != 0) fail(h, STAB_ERR_NUMERIC, "IRAM: Hessenberg QR failed");
      for (int i = 0; i < m; ++i) order[i] = i;
      auto lam_of = [&](cd t) { return (sigma * t - tau) / (t - 1.0); };
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        double aa = std::abs(theta[a]), ab = std::abs(theta[b]);
        if (aa != ab) return aa > ab;
        cd la = lam_of(theta[a]), lb = lam_of(theta[b]);
        if (la.real() != lb.real()) return la.real() > lb.real();
        return la.imag() > lb.imag();
      });
      double hn = 0.0;
      for (auto& z : H) hn += std::norm(z);
      hn = std::sqrt(hn);
      conv_count = 0;
      for (int q = 0; q < k; ++q) {
        const int i = order[q];
        est[q] = fnorm * std::abs(Y[(size_t)(m - 1) * m + i]);
        if (est[q] <= std::max(2.220446049250313e-16 * hn, tol * std::abs(theta[i]))) ++conv_count;
      }
      if (conv_count == k || restart >= h->opts.max_restarts) {
        if (conv_count < k) { result = STAB_ERR_NOT_CONVERGED; h->err = "stab_eigs: IRAM restart limit reached"; }
        break;
      }
      h->stats.restarts++;
      // exact shifts: the m - k unwanted Ritz values
      std::fill(Q.begin(), Q.end(), cd(0.0));
      for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
      for (int q = k; q < m; ++q) hess::shifted_qr(m, H.data(), Q.data(), theta[order[q]]);
      const cd beta_k = H[(size_t)k * m + k - 1];
      const cd sig_k = Q[(size_t)(m - 1) * m + k - 1];
      // tmp = V Q[:, 0:k+1];  f = tmp_k beta_k + f sigma_k;  V[:, 0:k] = tmp[:, 0:k]
      std::vector<cd> Qc((size_t)m * (k + 1));
      for (int jj = 0; jj <= k; ++jj)
        for (int l = 0; l < m; ++l) Qc[(size_t)jj * m + l] = Q[(size_t)l * m + jj];
      ck(h, cudaMemcpyAsync(dQ, Qc.data(), sizeof(double2) * Qc.size(), cudaMemcpyHostToDevice, h->stream), "copy Q");
      ck(h, kry_update_basis(h, V, m, k + 1, n, dQ, tmp), "V Q");
      ck(h, kry_axpby(h, d2(beta_k), tmp + (size_t)k * n, d2(sig_k), f, n), "f update");
      ck(h, cudaMemcpyAsync(V, tmp, sizeof(double2) * (size_t)k * n, cudaMemcpyDeviceToDevice, h->stream), "copy V");
      ck(h, cudaStreamSynchronize(h->stream), "sync");
      for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c)
          if (r >= k || c >= k) H[(size_t)r * m + c] = 0.0;
      j0 = k;
    }
    // eigenpairs: x_q = V y_q, lambda_q = (sigma theta - tau)/(theta - 1)
    std::vector<cd> Yw((size_t)m * k);
    for (int q = 0; q < k; ++q)
      for (int l = 0; l < m; ++l) Yw[(size_t)q * m + l] = Y[(size_t)l * m + order[q]];
    ck(h, cudaMemcpyAsync(dQ, Yw.data(), sizeof(double2) * Yw.size(), cudaMemcpyHostToDevice, h->stream), "copy Y");
    double2* X = tmp;  // k vectors (tmp holds k + 1)
    ck(h, kry_update_basis(h, V, m, k, n, dQ, X), "V Y");
    for (int q = 0; q < k; ++q) {
      const cd t = theta[order[q]];
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
