// CPU oracle for the stability path -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow restatement of the discretised right-hand side N(q) of the
// compressible Navier-Stokes equations in primitive (p, u_i, s) form
// (Sec. "Governing equations", Eq. navier_stokes) and of the matrix-free
// linearisation J(q0) v (Sec. "Matrix free framework", Eq. frechet).
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may
// load this library.  It shares no code with the CUDA library.
//
// Every routine is templated on the scalar type T so the same text is
// evaluated in double, in binary128 ("quad", for the exact value of the
// epsilon-quotient) and in std::complex<double> (complex-step tangent).
//
// Readings taken where the paper is silent or garbled (each listed in the
// design notes):
//  * the pressure equation carries the convective term u_j dp/dx_j;
//  * the entropy source is +(1/(rho T)) (div(lambda grad T) + Phi);
//  * nondimensionalisation by delta, u_inf, rho_inf: p_ref = 1/(gamma Ma^2),
//    T_ref = 1, R = p_ref, c_v = R/(gamma-1), c_p = gamma R/(gamma-1),
//    s = c_v ln(p/p_ref) - c_p ln(rho), mu = (1/Re) T^1.5 (1+S)/(T+S),
//    lambda = mu c_p / Pr, bulk viscosity mu_v = bulk * mu;
//  * "sixth order compact on a staggered grid" -> Lele's collocated 6th-order
//    tridiagonal schemes (first: alpha=1/3, a=14/9, b=1/9; second:
//    alpha=2/11, a=12/11, b=3/11); "fifth order" dissipation -> the compact
//    second derivative; bounded-direction closures: 3rd-order one-sided row
//    at the wall points and the 4th-order Pade row next to them;
//  * non-reflective y boundaries: LODI-type wave amplitudes
//    X+- = (v +- c)(dp/dy +- rho c dv/dy)/2 with incoming amplitudes removed,
//    the incoming/outgoing decision frozen on the base state.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 quad;
static inline quad o_exp(quad x) { return expq(x); }
static inline quad o_log(quad x) { return logq(x); }
static inline quad o_sqrt(quad x) { return sqrtq(x); }
static inline quad o_pow(quad x, double e) { return powq(x, (quad)e); }
#elif defined(__aarch64__)
typedef long double quad;  // IEEE binary128 on AArch64 Linux
static inline quad o_exp(quad x) { return expl(x); }
static inline quad o_log(quad x) { return logl(x); }
static inline quad o_sqrt(quad x) { return sqrtl(x); }
static inline quad o_pow(quad x, double e) { return powl(x, (quad)e); }
#else
#error "binary128 support required"
#endif

typedef std::complex<double> cplx;
static inline double o_exp(double x) { return std::exp(x); }
static inline double o_log(double x) { return std::log(x); }
static inline double o_sqrt(double x) { return std::sqrt(x); }
static inline double o_pow(double x, double e) { return std::pow(x, e); }
static inline cplx o_exp(cplx x) { return std::exp(x); }
static inline cplx o_log(cplx x) { return std::log(x); }
static inline cplx o_sqrt(cplx x) { return std::sqrt(x); }
static inline cplx o_pow(cplx x, double e) { return std::exp(e * std::log(x)); }

extern "C" {
// Problem description, laid out for ctypes.
struct OrcProblem {
  int dim, nx, ny, nz;
  double lx, ly0, ly1, lz, stretch;
  double gamma, Ma, Re, Pr, S, bulk;
  int low_order;  // 1: the reduced operator (second-order explicit differences)
};
}

// ---------------------------------------------------------------------------
// Tridiagonal solvers (textbook Thomas elimination; the cyclic case by the
// Sherman-Morrison formula).  Row i reads a[i] x[i-1] + b[i] x[i] + c[i] x[i+1].
// ---------------------------------------------------------------------------
template <class T>
static void thomas(const std::vector<double>& a, const std::vector<double>& b,
                   const std::vector<double>& c, std::vector<T>& d) {
  const int n = (int)d.size();
  std::vector<double> cp(n);
  std::vector<T> dp(n);
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; ++i) {
    double m = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / m;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / m;
  }
  d[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) d[i] = dp[i] - cp[i] * d[i + 1];
}

// Cyclic tridiagonal: a[0] multiplies x[n-1], c[n-1] multiplies x[0].
template <class T>
static void thomas_cyclic(const std::vector<double>& a, const std::vector<double>& b,
                          const std::vector<double>& c, std::vector<T>& d) {
  const int n = (int)d.size();
  const double alpha = c[n - 1];  // bottom-left corner
  const double beta = a[0];       // top-right corner
  const double g = -b[0];
  std::vector<double> bb(b);
  bb[0] = b[0] - g;
  bb[n - 1] = b[n - 1] - alpha * beta / g;
  std::vector<double> aa(a), cc(c);
  aa[0] = 0.0;
  cc[n - 1] = 0.0;
  std::vector<T> x(d);
  thomas(aa, bb, cc, x);
  std::vector<double> u(n, 0.0);
  u[0] = g;
  u[n - 1] = alpha;
  std::vector<double> z(u);
  thomas(aa, bb, cc, z);
  T fact = (x[0] + (beta / g) * x[n - 1]) / (1.0 + z[0] + (beta / g) * z[n - 1]);
  for (int i = 0; i < n; ++i) d[i] = x[i] - fact * z[i];
}

// ---------------------------------------------------------------------------
// Compact finite differences on one grid line (Lele 1992), spacing h.
// ---------------------------------------------------------------------------
// First derivative, periodic line: alpha f'_{i-1} + f'_i + alpha f'_{i+1}
//   = a (f_{i+1}-f_{i-1})/(2h) + b (f_{i+2}-f_{i-2})/(4h).
template <class T>
static void d1_periodic(const std::vector<T>& f, std::vector<T>& out, double h) {
  const int n = (int)f.size();
  const double al = 1.0 / 3.0, a = 14.0 / 9.0, b = 1.0 / 9.0;
  out.assign(n, T(0));
  for (int i = 0; i < n; ++i) {
    int ip1 = (i + 1) % n, im1 = (i - 1 + n) % n, ip2 = (i + 2) % n, im2 = (i - 2 + 2 * n) % n;
    out[i] = a * (f[ip1] - f[im1]) / (2.0 * h) + b * (f[ip2] - f[im2]) / (4.0 * h);
  }
  std::vector<double> A(n, al), B(n, 1.0), C(n, al);
  thomas_cyclic(A, B, C, out);
}

// Second derivative, periodic line: alpha f''_{i-1} + f''_i + alpha f''_{i+1}
//   = a (f_{i+1}-2f_i+f_{i-1})/h^2 + b (f_{i+2}-2f_i+f_{i-2})/(4h^2).
template <class T>
static void d2_periodic(const std::vector<T>& f, std::vector<T>& out, double h) {
  const int n = (int)f.size();
  const double al = 2.0 / 11.0, a = 12.0 / 11.0, b = 3.0 / 11.0;
  out.assign(n, T(0));
  for (int i = 0; i < n; ++i) {
    int ip1 = (i + 1) % n, im1 = (i - 1 + n) % n, ip2 = (i + 2) % n, im2 = (i - 2 + 2 * n) % n;
    out[i] = a * (f[ip1] - 2.0 * f[i] + f[im1]) / (h * h) +
             b * (f[ip2] - 2.0 * f[i] + f[im2]) / (4.0 * h * h);
  }
  std::vector<double> A(n, al), B(n, 1.0), C(n, al);
  thomas_cyclic(A, B, C, out);
}

// First derivative, bounded line (n >= 6).  Rows 0 and n-1: third-order
// one-sided  f'_0 + 2 f'_1 = (-5/2 f_0 + 2 f_1 + 1/2 f_2)/h  (mirrored with a
// sign change at the far end).  Rows 1 and n-2: fourth-order Pade
// f'_{i-1}/4 + f'_i + f'_{i+1}/4 = (3/2)(f_{i+1}-f_{i-1})/(2h).  Interior: the
// sixth-order scheme above.
template <class T>
static void d1_bounded(const std::vector<T>& f, std::vector<T>& out, double h) {
  const int n = (int)f.size();
  const double al = 1.0 / 3.0, a = 14.0 / 9.0, b = 1.0 / 9.0;
  std::vector<double> A(n, al), B(n, 1.0), C(n, al);
  out.assign(n, T(0));
  for (int i = 2; i < n - 2; ++i)
    out[i] = a * (f[i + 1] - f[i - 1]) / (2.0 * h) + b * (f[i + 2] - f[i - 2]) / (4.0 * h);
  A[0] = 0.0; C[0] = 2.0;
  out[0] = (-2.5 * f[0] + 2.0 * f[1] + 0.5 * f[2]) / h;
  A[n - 1] = 2.0; C[n - 1] = 0.0;
  out[n - 1] = -(-2.5 * f[n - 1] + 2.0 * f[n - 2] + 0.5 * f[n - 3]) / h;
  A[1] = 0.25; C[1] = 0.25;
  out[1] = 1.5 * (f[2] - f[0]) / (2.0 * h);
  A[n - 2] = 0.25; C[n - 2] = 0.25;
  out[n - 2] = 1.5 * (f[n - 1] - f[n - 3]) / (2.0 * h);
  thomas(A, B, C, out);
}

// Second derivative, bounded line (n >= 6).  Rows 0 and n-1: third-order
// one-sided  f''_0 + 11 f''_1 = (13 f_0 - 27 f_1 + 15 f_2 - f_3)/h^2 (mirrored).
// Rows 1 and n-2: fourth-order Pade
// f''_{i-1}/10 + f''_i + f''_{i+1}/10 = (6/5)(f_{i+1}-2f_i+f_{i-1})/h^2.
template <class T>
static void d2_bounded(const std::vector<T>& f, std::vector<T>& out, double h) {
  const int n = (int)f.size();
  const double al = 2.0 / 11.0, a = 12.0 / 11.0, b = 3.0 / 11.0;
  const double h2 = h * h;
  std::vector<double> A(n, al), B(n, 1.0), C(n, al);
  out.assign(n, T(0));
  for (int i = 2; i < n - 2; ++i)
    out[i] = a * (f[i + 1] - 2.0 * f[i] + f[i - 1]) / h2 + b * (f[i + 2] - 2.0 * f[i] + f[i - 2]) / (4.0 * h2);
  A[0] = 0.0; C[0] = 11.0;
  out[0] = (13.0 * f[0] - 27.0 * f[1] + 15.0 * f[2] - f[3]) / h2;
  A[n - 1] = 11.0; C[n - 1] = 0.0;
  out[n - 1] = (13.0 * f[n - 1] - 27.0 * f[n - 2] + 15.0 * f[n - 3] - f[n - 4]) / h2;
  A[1] = 0.1; C[1] = 0.1;
  out[1] = 1.2 * (f[2] - 2.0 * f[1] + f[0]) / h2;
  A[n - 2] = 0.1; C[n - 2] = 0.1;
  out[n - 2] = 1.2 * (f[n - 1] - 2.0 * f[n - 2] + f[n - 3]) / h2;
  thomas(A, B, C, out);
}

// ---------------------------------------------------------------------------
// Reduced operator (Sec. "Numerical experiments", the proposed preconditioner
// operator: a non-compact, lower-order discretisation of N).  Second-order
// explicit central differences, f'_i = (f_{i+1} - f_{i-1})/(2h) and
// f''_i = (f_{i+1} - 2 f_i + f_{i-1})/h^2; on a bounded line the end rows use
// the second-order one-sided forms f'_0 = (-3 f_0 + 4 f_1 - f_2)/(2h) and
// f''_0 = (2 f_0 - 5 f_1 + 4 f_2 - f_3)/h^2 (mirrored, the first with a sign
// change, at the far end).
// ---------------------------------------------------------------------------
template <class T>
static void low_line(const std::vector<T>& f, std::vector<T>& out, double h, int order, bool periodic) {
  const int n = (int)f.size();
  out.assign(n, T(0));
  for (int i = 0; i < n; ++i) {
    int ip = i + 1, im = i - 1;
    if (periodic) { ip %= n; im = (im + n) % n; }
    else if (i == 0 || i == n - 1) continue;
    out[i] = order == 1 ? (f[ip] - f[im]) / (2.0 * h) : (f[ip] - 2.0 * f[i] + f[im]) / (h * h);
  }
  if (periodic) return;
  const int e = n - 1;
  if (order == 1) {
    out[0] = (-3.0 * f[0] + 4.0 * f[1] - f[2]) / (2.0 * h);
    out[e] = (3.0 * f[e] - 4.0 * f[e - 1] + f[e - 2]) / (2.0 * h);
  } else {
    out[0] = (2.0 * f[0] - 5.0 * f[1] + 4.0 * f[2] - f[3]) / (h * h);
    out[e] = (2.0 * f[e] - 5.0 * f[e - 1] + 4.0 * f[e - 2] - f[e - 3]) / (h * h);
  }
}

// ---------------------------------------------------------------------------
// Grid fields and derivatives along an axis (0 = x, 1 = y, 2 = z).
// Arrays are [z][y][x], x fastest.
// ---------------------------------------------------------------------------
struct Geo {
  int nx, ny, nz, dim, low;
  double hx, hz, heta;
  std::vector<double> yp, ypp;  // dy/deta, d2y/deta2 per y row
};

static Geo make_geo(const OrcProblem& P) {
  Geo g;
  g.nx = P.nx; g.ny = P.ny; g.nz = P.nz; g.dim = P.dim; g.low = P.low_order;
  g.hx = P.lx / P.nx;
  g.hz = P.dim == 3 ? P.lz / P.nz : 1.0;
  g.heta = 1.0 / (P.ny - 1);
  g.yp.resize(P.ny);
  g.ypp.resize(P.ny);
  for (int j = 0; j < P.ny; ++j) {
    double eta = j * g.heta;
    if (P.stretch == 0.0) {
      g.yp[j] = P.ly1 - P.ly0;
      g.ypp[j] = 0.0;
    } else {
      // y(eta) = yc + half sinh(beta (2 eta - 1)) / sinh(beta)
      double be = P.stretch, half = 0.5 * (P.ly1 - P.ly0), sb = std::sinh(be);
      g.yp[j] = half * 2.0 * be * std::cosh(be * (2.0 * eta - 1.0)) / sb;
      g.ypp[j] = half * 4.0 * be * be * std::sinh(be * (2.0 * eta - 1.0)) / sb;
    }
  }
  return g;
}

// order 1 or 2 derivative of field f along axis; y uses the stretching metric
// f_y = f_eta / y',  f_yy = f_etaeta / y'^2 - y'' f_eta / y'^3.
template <class T>
static std::vector<T> deriv(const Geo& g, const std::vector<T>& f, int axis, int order) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  std::vector<T> out(f.size());
  int nline, len;
  if (axis == 0) { len = nx; nline = ny * nz; }
  else if (axis == 1) { len = ny; nline = nx * nz; }
  else { len = nz; nline = nx * ny; }
#pragma omp parallel for schedule(static) if (nline >= 64)
  for (int L = 0; L < nline; ++L) {
    std::vector<T> line(len), d1, d2;
    auto idx = [&](int k) -> size_t {
      if (axis == 0) { int j = L % ny, kz = L / ny; return ((size_t)kz * ny + j) * nx + k; }
      if (axis == 1) { int i = L % nx, kz = L / nx; return ((size_t)kz * ny + k) * nx + i; }
      int i = L % nx, j = L / nx; return ((size_t)k * ny + j) * nx + i;
    };
    for (int k = 0; k < len; ++k) line[k] = f[idx(k)];
    if (axis == 0 || axis == 2) {
      double h = axis == 0 ? g.hx : g.hz;
      if (g.low) low_line(line, d1, h, order, true);
      else if (order == 1) d1_periodic(line, d1, h); else d2_periodic(line, d1, h);
      for (int k = 0; k < len; ++k) out[idx(k)] = d1[k];
    } else {
      if (g.low) low_line(line, d1, g.heta, 1, false); else d1_bounded(line, d1, g.heta);
      if (order == 1) {
        for (int k = 0; k < len; ++k) out[idx(k)] = d1[k] / g.yp[k];
      } else {
        if (g.low) low_line(line, d2, g.heta, 2, false); else d2_bounded(line, d2, g.heta);
        for (int k = 0; k < len; ++k)
          out[idx(k)] = d2[k] / (g.yp[k] * g.yp[k]) - g.ypp[k] * d1[k] / (g.yp[k] * g.yp[k] * g.yp[k]);
      }
    }
  }
  return out;
}

// ---------------------------------------------------------------------------
// The right-hand side N(q).  q0sw is the base state that freezes the
// incoming/outgoing decision at the non-reflective y boundaries.
// ---------------------------------------------------------------------------
template <class T>
static void rhs(const OrcProblem& P, const double* q0sw, const T* q, T* out) {
  const Geo g = make_geo(P);
  const int D = P.dim;
  const size_t N = (size_t)P.nx * P.ny * P.nz;
  const double gam = P.gamma;
  const double R = 1.0 / (gam * P.Ma * P.Ma);
  const double pref = R;
  const double cp = gam * R / (gam - 1.0);
  const bool visc = P.Re > 0.0;

  std::vector<T> p(q, q + N), s(q + (D + 1) * N, q + (D + 2) * N);
  std::vector<std::vector<T>> u(D);
  for (int i = 0; i < D; ++i) u[i].assign(q + (1 + i) * N, q + (2 + i) * N);

  // closure: rho(p, s) from s = c_v ln(p/p_ref) - c_p ln(rho); ideal gas T.
  std::vector<T> rho(N), Tm(N);
  for (size_t k = 0; k < N; ++k) {
    rho[k] = o_pow(p[k] / pref, 1.0 / gam) * o_exp(-s[k] / cp);
    Tm[k] = p[k] / (rho[k] * R);
  }

  // first derivatives dp[j], du[i][j] = d u_i / d x_j, ds[j], dT[j]
  std::vector<std::vector<T>> dp(D), ds(D), dT(D);
  std::vector<std::vector<std::vector<T>>> du(D, std::vector<std::vector<T>>(D));
  for (int j = 0; j < D; ++j) {
    dp[j] = deriv(g, p, j, 1);
    ds[j] = deriv(g, s, j, 1);
    for (int i = 0; i < D; ++i) du[i][j] = deriv(g, u[i], j, 1);
    if (visc) dT[j] = deriv(g, Tm, j, 1);
  }
  // second derivatives d2u[i][j] = d^2 u_i/dx_j^2, d2T[j]; mixed
  // mix[i][k] = d/dx_i (d u_k / dx_k) for i != k.
  std::vector<std::vector<std::vector<T>>> d2u(D, std::vector<std::vector<T>>(D));
  std::vector<std::vector<T>> d2T(D);
  std::vector<std::vector<std::vector<T>>> mix(D, std::vector<std::vector<T>>(D));
  if (visc) {
    for (int j = 0; j < D; ++j) {
      d2T[j] = deriv(g, Tm, j, 2);
      for (int i = 0; i < D; ++i) d2u[i][j] = deriv(g, u[i], j, 2);
    }
    for (int i = 0; i < D; ++i)
      for (int k = 0; k < D; ++k)
        if (i != k) mix[i][k] = deriv(g, du[k][k], i, 1);
  }

  T* pt = out;
  T* st = out + (D + 1) * N;
  const int Y = 1;  // y axis and index of the y velocity
#pragma omp parallel for schedule(static) if (N >= 4096)
  for (size_t k = 0; k < N; ++k) {
    const int jrow = (int)((k / P.nx) % P.ny);
    T div = T(0);
    for (int i = 0; i < D; ++i) div += du[i][i][k];

    T heat = T(0), Phi = T(0);
    std::vector<T> vis(D, T(0));
    if (visc) {
      T Tk = Tm[k];
      T mu = (1.0 / P.Re) * o_pow(Tk, 1.5) * (1.0 + P.S) / (Tk + P.S);
      T dmu = mu * (1.5 / Tk - 1.0 / (Tk + P.S));  // d mu / d T
      T lam = mu * cp / P.Pr, dlam = dmu * cp / P.Pr;
      T muv = P.bulk * mu, dmuv = P.bulk * dmu;
      T lapT = T(0), gT2 = T(0);
      for (int j = 0; j < D; ++j) { lapT += d2T[j][k]; gT2 += dT[j][k] * dT[j][k]; }
      heat = lam * lapT + dlam * gT2;
      T SS = T(0);
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          T sij = 0.5 * (du[i][j][k] + du[j][i][k]);
          SS += sij * sij;
        }
      Phi = 2.0 * mu * (SS - div * div / 3.0) + muv * div * div;
      for (int i = 0; i < D; ++i) {
        T lap = T(0), ddiv = T(0);
        for (int j = 0; j < D; ++j) lap += d2u[i][j][k];
        for (int kk = 0; kk < D; ++kk) ddiv += (kk == i) ? d2u[i][i][k] : mix[i][kk][k];
        T cross = T(0);
        for (int j = 0; j < D; ++j) cross += dmu * dT[j][k] * (du[i][j][k] + du[j][i][k]);
        vis[i] = mu * (lap + ddiv / 3.0) + muv * ddiv + cross + (dmuv - 2.0 / 3.0 * dmu) * dT[i][k] * div;
      }
    }

    // y-direction inviscid terms, possibly replaced at the y boundaries
    T yp_term = -(u[Y][k] * dp[Y][k] + gam * p[k] * du[Y][Y][k]);
    T yv_term = -(u[Y][k] * du[Y][Y][k] + dp[Y][k] / rho[k]);
    bool drop_conv = false;
    if (jrow == 0 || jrow == P.ny - 1) {
      const size_t Nsz = N;
      double p0 = q0sw[k], s0 = q0sw[(D + 1) * Nsz + k], v0 = q0sw[(1 + Y) * Nsz + k];
      double rho0 = std::pow(p0 / pref, 1.0 / gam) * std::exp(-s0 / cp);
      double c0 = std::sqrt(gam * p0 / rho0);
      bool top = (jrow == P.ny - 1);
      bool in_plus = top ? (v0 + c0 < 0.0) : (v0 + c0 > 0.0);
      bool in_minus = top ? (v0 - c0 < 0.0) : (v0 - c0 > 0.0);
      drop_conv = top ? (v0 < 0.0) : (v0 > 0.0);
      T c = o_sqrt(gam * p[k] / rho[k]);
      T rc = rho[k] * c;
      T Xp = 0.5 * (u[Y][k] + c) * (dp[Y][k] + rc * du[Y][Y][k]);
      T Xm = 0.5 * (u[Y][k] - c) * (dp[Y][k] - rc * du[Y][Y][k]);
      if (in_plus) Xp = T(0);
      if (in_minus) Xm = T(0);
      yp_term = -(Xp + Xm);
      yv_term = -(Xp - Xm) / rc;
    }

    // pressure: dp/dt = -u_j dp/dx_j - rho c^2 div u + (gamma-1)(heat + Phi), rho c^2 = gamma p
    T ptk = yp_term;
    for (int j = 0; j < D; ++j)
      if (j != Y) ptk -= u[j][k] * dp[j][k] + gam * p[k] * du[j][j][k];
    ptk += (gam - 1.0) * (heat + Phi);
    pt[k] = ptk;

    // velocities: du_i/dt = -u_j du_i/dx_j - (1/rho) dp/dx_i + (1/rho) d tau_ij/dx_j
    for (int i = 0; i < D; ++i) {
      T r = T(0);
      if (i == Y) {
        r = yv_term;
        for (int j = 0; j < D; ++j)
          if (j != Y) r -= u[j][k] * du[i][j][k];
      } else {
        for (int j = 0; j < D; ++j) {
          if (j == Y && drop_conv) continue;
          r -= u[j][k] * du[i][j][k];
        }
        r -= dp[i][k] / rho[k];
      }
      r += vis[i] / rho[k];
      out[(1 + i) * N + k] = r;
    }

    // entropy: ds/dt = -u_j ds/dx_j + (1/(rho T)) (heat + Phi), 1/(rho T) = R/p
    T stk = T(0);
    for (int j = 0; j < D; ++j) {
      if (j == Y && drop_conv) continue;
      stk -= u[j][k] * ds[j][k];
    }
    stk += (R / p[k]) * (heat + Phi);
    st[k] = stk;
  }
}

static size_t n_dofs(const OrcProblem& P) { return (size_t)(P.dim + 2) * P.nx * P.ny * P.nz; }

extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// One compact derivative of a single line (order 1 or 2; periodic or bounded).
void orc_deriv_line(int order, int periodic, int n, double h, const double* f, double* out) {
  std::vector<double> line(f, f + n), d;
  if (periodic) { if (order == 1) d1_periodic(line, d, h); else d2_periodic(line, d, h); }
  else { if (order == 1) d1_bounded(line, d, h); else d2_bounded(line, d, h); }
  std::memcpy(out, d.data(), sizeof(double) * n);
}

// One second-order explicit derivative of a single line (the reduced operator).
void orc_deriv_line_low(int order, int periodic, int n, double h, const double* f, double* out) {
  std::vector<double> line(f, f + n), d;
  low_line(line, d, h, order, periodic != 0);
  std::memcpy(out, d.data(), sizeof(double) * n);
}

// Derivative of a full grid field along an axis, including the y metric.
void orc_deriv_field(const OrcProblem* P, const double* f, int axis, int order, double* out) {
  Geo g = make_geo(*P);
  size_t N = (size_t)P->nx * P->ny * P->nz;
  std::vector<double> fv(f, f + N);
  std::vector<double> d = deriv(g, fv, axis, order);
  std::memcpy(out, d.data(), sizeof(double) * N);
}

// N(q) in double.
void orc_rhs(const OrcProblem* P, const double* q0sw, const double* q, double* out) {
  rhs<double>(*P, q0sw, q, out);
}

// N(q) in binary128 (input and output rounded through double).
void orc_rhs_quad(const OrcProblem* P, const double* q0sw, const double* q, double* out) {
  size_t n = n_dofs(*P);
  std::vector<quad> qq(q, q + n), oo(n);
  rhs<quad>(*P, q0sw, qq.data(), oo.data());
  for (size_t i = 0; i < n; ++i) out[i] = (double)oo[i];
}

// Literal epsilon-quotient (Eq. frechet) in double, for complex v
// (interleaved re/im): out = [N(q0 + eps Re v) - N(q0)]/eps + i [N(q0 + eps Im v) - N(q0)]/eps.
void orc_jv_literal(const OrcProblem* P, const double* q0, const double* v, double eps, double* out) {
  size_t n = n_dofs(*P);
  std::vector<double> base(n), qp(n), np(n);
  rhs<double>(*P, q0, q0, base.data());
  for (int part = 0; part < 2; ++part) {
    for (size_t i = 0; i < n; ++i) qp[i] = q0[i] + eps * v[2 * i + part];
    rhs<double>(*P, q0, qp.data(), np.data());
    for (size_t i = 0; i < n; ++i) out[2 * i + part] = (np[i] - base[i]) / eps;
  }
}

// The same quotient with every operation in binary128: the exact value of
// the quotient for this eps, to about 1e-25 relative.
void orc_jv_quad(const OrcProblem* P, const double* q0, const double* v, double eps, double* out) {
  size_t n = n_dofs(*P);
  std::vector<quad> q0q(n), qp(n), base(n), np(n);
  for (size_t i = 0; i < n; ++i) q0q[i] = q0[i];
  rhs<quad>(*P, q0, q0q.data(), base.data());
  quad e = eps;
  for (int part = 0; part < 2; ++part) {
    for (size_t i = 0; i < n; ++i) qp[i] = q0q[i] + e * (quad)v[2 * i + part];
    rhs<quad>(*P, q0, qp.data(), np.data());
    for (size_t i = 0; i < n; ++i) out[2 * i + part] = (double)((np[i] - base[i]) / e);
  }
}

// Exact tangent J(q0) v by the complex step: Im N(q0 + i h v)/h, h = 1e-30,
// applied to Re v and Im v separately.
void orc_jv_tangent(const OrcProblem* P, const double* q0, const double* v, double* out) {
  size_t n = n_dofs(*P);
  const double h = 1e-30;
  std::vector<cplx> qc(n), oc(n);
  for (int part = 0; part < 2; ++part) {
    for (size_t i = 0; i < n; ++i) qc[i] = cplx(q0[i], h * v[2 * i + part]);
    rhs<cplx>(*P, q0, qc.data(), oc.data());
    for (size_t i = 0; i < n; ++i) out[2 * i + part] = oc[i].imag() / h;
  }
}

// Dense tangent Jacobian, column-major (J[col * n + row]), column k = J e_k.
void orc_dense_jacobian(const OrcProblem* P, const double* q0, double* J) {
  const long n = (long)n_dofs(*P);
  const double h = 1e-30;
#pragma omp parallel
  {
    std::vector<cplx> qc(n), oc(n);
#pragma omp for schedule(dynamic, 4)
    for (long col = 0; col < n; ++col) {
      for (long i = 0; i < n; ++i) qc[i] = cplx(q0[i], 0.0);
      qc[col] = cplx(q0[col], h);
      rhs<cplx>(*P, q0, qc.data(), oc.data());
      for (long i = 0; i < n; ++i) J[col * n + i] = oc[i].imag() / h;
    }
  }
}

// Selected columns of the dense tangent Jacobian (cols[k] -> J[:, k]).
void orc_jacobian_columns(const OrcProblem* P, const double* q0, const long* cols, long ncols, double* J) {
  const long n = (long)n_dofs(*P);
  const double h = 1e-30;
#pragma omp parallel
  {
    std::vector<cplx> qc(n), oc(n);
#pragma omp for schedule(dynamic, 1)
    for (long c = 0; c < ncols; ++c) {
      for (long i = 0; i < n; ++i) qc[i] = cplx(q0[i], 0.0);
      qc[cols[c]] = cplx(q0[cols[c]], h);
      rhs<cplx>(*P, q0, qc.data(), oc.data());
      for (long i = 0; i < n; ++i) J[c * n + i] = oc[i].imag() / h;
    }
  }
}

}  // extern "C"
