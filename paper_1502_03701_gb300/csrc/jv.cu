// Matrix-free J(q0) v of the discretised compressible Navier-Stokes
// right-hand side (Eq. navier_stokes, linearised by Eq. frechet).
//
// Pipeline per call (all on the handle's stream):
//   1. eps: ||v||_2 by a fixed-order two-stage reduction, then
//      eps = sqrt(eps_m)(1 + ||q0||)/||v|| (or the fixed / zero value);
//   2. Tw  : the scaled temperature difference [T(q0 + eps v) - T(q0)]/eps,
//            pointwise and free of cancellation;
//   3. line passes y, (z), x: compact first / second / mixed derivatives of
//      the scaled differences (derivatives are linear, so
//      D[f(q0 + eps v)] - D[f(q0)] = D[f(q0 + eps v) - f(q0)]);
//   4. pointwise assembly of [N(q0 + eps v) - N(q0)]/eps in
//      difference-number arithmetic, minus shift * v.
// With eps = 0 the same arithmetic yields the exact tangent J(q0) v.
#include <cfloat>
#include <cmath>

#include "internal.cuh"

namespace {

// ---------------------------------------------------------------------------
// Difference numbers: a = base value, w = (perturbed - base)/eps.  Every
// operation below is an exact identity for the scaled difference, so the
// quotient is formed without subtracting nearly equal numbers.
// ---------------------------------------------------------------------------
struct DN {
  double a, w;
};
__device__ __forceinline__ DN dn(double a, double w) { return DN{a, w}; }
__device__ __forceinline__ DN operator+(DN x, DN y) { return dn(x.a + y.a, x.w + y.w); }
__device__ __forceinline__ DN operator-(DN x, DN y) { return dn(x.a - y.a, x.w - y.w); }
__device__ __forceinline__ DN operator-(DN x) { return dn(-x.a, -x.w); }
__device__ __forceinline__ DN operator*(double c, DN x) { return dn(c * x.a, c * x.w); }
__device__ __forceinline__ DN add(DN x, double c) { return dn(x.a + c, x.w); }
// (a1 + e w1)(a2 + e w2) - a1 a2 = e [a1 w2 + w1 (a2 + e w2)]
__device__ __forceinline__ DN mul(DN x, DN y, double e) {
  return dn(x.a * y.a, fma(x.a, y.w, x.w * fma(e, y.w, y.a)));
}
// 1/(a + e w) - 1/a = -e w / (a (a + e w))
__device__ __forceinline__ DN rcp(DN x, double e) {
  double inv = 1.0 / x.a;
  return dn(inv, -x.w / (x.a * fma(e, x.w, x.a)));
}
// sqrt(a + e w) - sqrt(a) = e w / (sqrt(a + e w) + sqrt(a))
__device__ __forceinline__ DN dsqrt(DN x, double e) {
  double s = sqrt(x.a);
  return dn(s, x.w / (sqrt(fma(e, x.w, x.a)) + s));
}
// expm1(z)/z and log1p(z)/z with their limits at z = 0
__device__ __forceinline__ double expm1_over(double z) { return z == 0.0 ? 1.0 : expm1(z) / z; }
__device__ __forceinline__ double log1p_over(double z) { return z == 0.0 ? 1.0 : log1p(z) / z; }

// Scaled differences of the closure rho(p, s) = (p/p_ref)^{1/gamma} e^{-s/c_p}
// and T(p, s) = (p/p_ref)^{(gamma-1)/gamma} e^{s/c_p}:
//   rho(q0 + e w)/rho0 = exp(x_rho),  x_rho = (1/gamma) log1p(e wp/p0) - e ws/c_p.
struct ClosureK {
  double ig, omig, icp;  // 1/gamma, 1 - 1/gamma, 1/c_p
};
__device__ __forceinline__ void closure_w(const ClosureK& C, double p0, double rho0, double T0, double wp,
                                          double ws, double e, double* wrho, double* wT) {
  double q = wp / p0;
  double lq = q * log1p_over(e * q);
  double xr = C.ig * lq - ws * C.icp;
  double xt = C.omig * lq + ws * C.icp;
  if (wrho) *wrho = rho0 * expm1_over(e * xr) * xr;
  if (wT) *wT = T0 * expm1_over(e * xt) * xt;
}

// ---------------------------------------------------------------------------
// Base-table layout (real arrays of length nbase, physical derivatives).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int bt_val(int D, int f) { (void)D; return f; }  // p,u..,s,T,rho
__host__ __device__ __forceinline__ int bt_d1(int D, int ax, int f) { return (D + 4) + ax * (D + 3) + f; }
__host__ __device__ __forceinline__ int bt_d2(int D, int ax, int g) { return (D + 4) + D * (D + 3) + ax * (D + 1) + g; }
__host__ __device__ __forceinline__ int bt_mix(int D, int i, int k) {
  return (D + 4) + D * (D + 3) + D * (D + 1) + i * D + k;
}
__host__ __device__ __forceinline__ int bt_count(int D) { return (D + 4) + D * (D + 3) + D * (D + 1) + D * D; }

// ---------------------------------------------------------------------------
// Line pass: compact derivatives along one axis for a batch of fields.
// A CTA stages L lines x n points of one field in shared memory; each thread
// runs one chunk of one line for one derivative kind, first forward (with a
// warm-up of K points, after which the influence of the unknown start value
// has decayed below 2^-56), then backward.
// ---------------------------------------------------------------------------
struct PassParams {
  LineJob job[STAB_MAX_JOBS];
  int njobs;
  int axis, n, nx, ny;
  long long nlines;
  long long stride;
  int L, C, nchunks;
  int periodic;
  double c1[2], c2[2];  // interior stencil weights per kind
  double h;
  const double* tab[2];
  int K[2];
};

__device__ __forceinline__ long long line_base(const PassParams& P, long long l) {
  if (P.axis == 0) return l * P.nx;
  if (P.axis == 1) return (l / P.nx) * (long long)P.nx * P.ny + (l % P.nx);
  return l;
}

__device__ __forceinline__ int wrapi(int t, int n) {
  int r = t % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ double2 d2sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 d2lin(double c1, double2 a, double c2, double2 b) {
  return make_double2(c1 * a.x + c2 * b.x, c1 * a.y + c2 * b.y);
}

// right-hand side B f of the compact scheme at point t
__device__ double2 stencil_rhs(const PassParams& P, const double2* F, int L, int lt, int t, int kind) {
  const int n = P.n;
  auto f = [&](int s) { return F[(P.periodic ? wrapi(s, n) : s) * L + lt]; };
  const double h = P.h;
  if (!P.periodic && (t < 2 || t > n - 3)) {
    if (kind == 0) {
      if (t == 0) { double2 a = f(0), b = f(1), c = f(2); return make_double2((-2.5 * a.x + 2.0 * b.x + 0.5 * c.x) / h, (-2.5 * a.y + 2.0 * b.y + 0.5 * c.y) / h); }
      if (t == n - 1) { double2 a = f(n - 1), b = f(n - 2), c = f(n - 3); return make_double2((2.5 * a.x - 2.0 * b.x - 0.5 * c.x) / h, (2.5 * a.y - 2.0 * b.y - 0.5 * c.y) / h); }
      double2 d = d2sub(f(t + 1), f(t - 1));
      return make_double2(0.75 * d.x / h, 0.75 * d.y / h);
    } else {
      const double ih2 = 1.0 / (h * h);
      if (t == 0 || t == n - 1) {
        int s = t == 0 ? 1 : -1;
        double2 a = f(t), b = f(t + s), c = f(t + 2 * s), d = f(t + 3 * s);
        return make_double2((13.0 * a.x - 27.0 * b.x + 15.0 * c.x - d.x) * ih2, (13.0 * a.y - 27.0 * b.y + 15.0 * c.y - d.y) * ih2);
      }
      double2 a = f(t - 1), b = f(t), c = f(t + 1);
      return make_double2(1.2 * (c.x - 2.0 * b.x + a.x) * ih2, 1.2 * (c.y - 2.0 * b.y + a.y) * ih2);
    }
  }
  double2 fm2 = f(t - 2), fm1 = f(t - 1), fp1 = f(t + 1), fp2 = f(t + 2);
  if (kind == 0) return d2lin(P.c1[0], d2sub(fp1, fm1), P.c2[0], d2sub(fp2, fm2));
  double2 f0 = f(t);
  double2 s1 = make_double2(fp1.x - 2.0 * f0.x + fm1.x, fp1.y - 2.0 * f0.y + fm1.y);
  double2 s2 = make_double2(fp2.x - 2.0 * f0.x + fm2.x, fp2.y - 2.0 * f0.y + fm2.y);
  return d2lin(P.c1[1], s1, P.c2[1], s2);
}

__global__ void k_line_pass(const PassParams P) {
  extern __shared__ double2 sm[];
  const LineJob J = P.job[blockIdx.y];
  const int n = P.n, L = P.L;
  double2* F = sm;
  double2* G[2] = {sm + (size_t)n * L, sm + (size_t)2 * n * L};
  const long long l0 = (long long)blockIdx.x * L;

  for (int idx = threadIdx.x; idx < n * L; idx += blockDim.x) {
    int lt, t;
    if (P.axis == 0) { lt = idx / n; t = idx % n; } else { t = idx / L; lt = idx % L; }
    long long l = l0 + lt;
    double2 val = make_double2(0.0, 0.0);
    if (l < P.nlines) val = J.in[line_base(P, l) + (long long)t * P.stride];
    F[t * L + lt] = val;
  }
  __syncthreads();

  const int per = L * P.nchunks;
  const int kind = threadIdx.x / per;
  const int rem = threadIdx.x % per;
  const int lt = rem % L, ch = rem / L;
  double2* out = kind == 0 ? J.out1 : J.out2;
  const bool active = kind < 2 && out != nullptr && (l0 + lt) < P.nlines;
  const int t0 = ch * P.C, t1 = min(n, t0 + P.C);
  const double* tl = P.tab[kind < 2 ? kind : 0];
  const double* tdinv = tl + n;
  const double* tm = tl + 2 * n;
  const int K = P.K[kind < 2 ? kind : 0];
  double2* Gk = G[kind < 2 ? kind : 0];

  if (active) {
    int ts = P.periodic ? t0 - K : ((t0 - K < 8) ? 0 : t0 - K);
    double2 g = make_double2(0.0, 0.0);
    for (int t = ts; t < t1; ++t) {
      int tt = P.periodic ? wrapi(t, n) : t;
      double2 r = stencil_rhs(P, F, L, lt, tt, kind);
      double lv = __ldg(tl + tt);
      g.x = fma(-lv, g.x, r.x);
      g.y = fma(-lv, g.y, r.y);
      if (t >= t0) Gk[tt * L + lt] = g;
    }
  }
  __syncthreads();
  if (active) {
    int te = P.periodic ? t1 - 1 + K : ((t1 - 1 + K > n - 9) ? n - 1 : t1 - 1 + K);
    double2 x = make_double2(0.0, 0.0);
    const long long base = line_base(P, l0 + lt);
    for (int t = te; t >= t0; --t) {
      int tt = P.periodic ? wrapi(t, n) : t;
      double2 gg = Gk[tt * L + lt];
      double di = __ldg(tdinv + tt), mm = __ldg(tm + tt);
      x.x = fma(gg.x, di, -mm * x.x);
      x.y = fma(gg.y, di, -mm * x.y);
      if (t < t1) out[base + (long long)tt * P.stride] = x;
    }
  }
}

// ---------------------------------------------------------------------------
// Reductions: ||v||^2 in a fixed order (deterministic), then epsilon.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__global__ void k_norm2_partial(const double2* __restrict__ v, long long n, double* partial) {
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 z = v[i];
    s = fma(z.x, z.x, fma(z.y, z.y, s));
  }
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

// mode 0: out = sum;  mode 1: out = sqrt(sum);  mode 2: epsilon from ||v||
__global__ void k_norm2_final(const double* partial, int nb, double* out, int mode, double q0norm, double fixed_eps) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += partial[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    if (mode == 0) *out = s;
    else if (mode == 1) *out = sqrt(s);
    else {
      double e = 0.0;
      if (fixed_eps > 0.0) e = fixed_eps;
      else if (s > 0.0) e = 1.4901161193847656e-08 * (1.0 + q0norm) / sqrt(s);  // sqrt(2^-52)
      *out = e;
    }
  }
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// ---------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------
struct PointParams {
  const double2* v;
  const double2* scratch;
  long long npts;
  int nx, ny, nz, D;
  int homog, visc;
  int s_Tw;
  int s_d1[3][6], s_d2[3][4], s_mix[3][3];
  const double* btab;
  long long nbase;
  const double* eta_y;
  const double* eta_yy;
  const unsigned char* bcflags;
  const double* eps;
  double2* out;
  double2 shift;
  double gamma, R, cp, Pr, S, Re, bulk;
  ClosureK C;
};

__global__ void k_temperature(const PointParams P, double2* Tw) {
  const int D = P.D;
  const double e = *P.eps;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)gridDim.x * blockDim.x) {
    int j = (int)((pt / P.nx) % P.ny);
    long long b = P.homog ? j : pt;
    double p0 = P.btab[bt_val(D, 0) * P.nbase + b];
    double T0 = P.btab[bt_val(D, D + 2) * P.nbase + b];
    double2 wp = P.v[pt], ws = P.v[(long long)(D + 1) * P.npts + pt];
    double t0, t1;
    closure_w(P.C, p0, 0.0, T0, wp.x, ws.x, e, nullptr, &t0);
    closure_w(P.C, p0, 0.0, T0, wp.y, ws.y, e, nullptr, &t1);
    Tw[pt] = make_double2(t0, t1);
  }
}

template <int D>
__device__ void point_rhs(const PointParams& P, long long pt, int i, int j, int k, int part, double e, double* res) {
  const long long b = P.homog ? j : pt;
  const double* BT = P.btab;
  const long long NB = P.nbase;
  auto B = [&](int slot) { return BT[(long long)slot * NB + b]; };
  auto Wv = [&](const double2* f) { double2 z = f[pt]; return part ? z.y : z.x; };
  auto S_ = [&](int slot) { return P.scratch + (long long)slot * P.npts; };
  const double ey = P.eta_y[j], eyy = P.eta_yy[j];
  const int Y = 1;

  DN p = dn(B(bt_val(D, 0)), Wv(P.v));
  DN u[D];
#pragma unroll
  for (int a = 0; a < D; ++a) u[a] = dn(B(bt_val(D, 1 + a)), Wv(P.v + (long long)(1 + a) * P.npts));
  DN s = dn(B(bt_val(D, D + 1)), Wv(P.v + (long long)(D + 1) * P.npts));
  const double T0 = B(bt_val(D, D + 2)), rho0 = B(bt_val(D, D + 3));
  double wrho;
  closure_w(P.C, p.a, rho0, T0, p.w, s.w, e, &wrho, nullptr);
  DN rho = dn(rho0, wrho);

  auto D1 = [&](int ax, int f) {
    double w = Wv(S_(P.s_d1[ax][f]));
    if (ax == Y) w *= ey;
    return dn(B(bt_d1(D, ax, f)), w);
  };
  DN dp[D], ds[D], du[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    dp[a] = D1(a, 0);
    ds[a] = D1(a, D + 1);
#pragma unroll
    for (int c = 0; c < D; ++c) du[c][a] = D1(a, 1 + c);
  }
  DN div = du[0][0];
#pragma unroll
  for (int a = 1; a < D; ++a) div = div + du[a][a];

  DN heat = dn(0.0, 0.0), Phi = dn(0.0, 0.0);
  DN vis[D];
#pragma unroll
  for (int a = 0; a < D; ++a) vis[a] = dn(0.0, 0.0);
  if (P.visc) {
    DN T = dn(T0, Wv(P.scratch + (long long)P.s_Tw * P.npts));
    DN dT[D];
#pragma unroll
    for (int a = 0; a < D; ++a) dT[a] = D1(a, D + 2);
    auto D2 = [&](int ax, int g, int f) {
      double w = Wv(S_(P.s_d2[ax][g]));
      if (ax == Y) w = fma(w, ey * ey, Wv(S_(P.s_d1[ax][f])) * eyy);
      return dn(B(bt_d2(D, ax, g)), w);
    };
    auto MX = [&](int a, int c) {
      double w = Wv(S_(P.s_mix[a][c]));
      if (a == Y || c == Y) w *= ey;
      return dn(B(bt_mix(D, a, c)), w);
    };
    // Sutherland: mu = (1+S)/Re T^{3/2}/(T+S);  dmu/dT = mu (3/(2T) - 1/(T+S))
    DN sqT = dsqrt(T, e);
    DN rTS = rcp(add(T, P.S), e);
    DN mu = ((1.0 + P.S) / P.Re) * mul(mul(T, sqT, e), rTS, e);
    DN dmu = mul(mu, 1.5 * rcp(T, e) - rTS, e);
    const double kl = P.cp / P.Pr;
    DN lam = kl * mu, dlam = kl * dmu;
    DN muv = P.bulk * mu, dmuv = P.bulk * dmu;
    DN lapT = dn(0.0, 0.0), gT2 = dn(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lapT = lapT + D2(a, D, D + 2);
      gT2 = gT2 + mul(dT[a], dT[a], e);
    }
    heat = mul(lam, lapT, e) + mul(dlam, gT2, e);
    DN SS = dn(0.0, 0.0);
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        DN sij = 0.5 * (du[a][c] + du[c][a]);
        SS = SS + mul(sij, sij, e);
      }
    DN div2 = mul(div, div, e);
    Phi = 2.0 * mul(mu, SS - (1.0 / 3.0) * div2, e) + mul(muv, div2, e);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      DN lap = dn(0.0, 0.0), ddiv = dn(0.0, 0.0), cross = dn(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        DN d2ac = D2(c, a, 1 + a);  // d^2 u_a / dx_c^2
        lap = lap + d2ac;
        ddiv = ddiv + (c == a ? d2ac : MX(a, c));
        cross = cross + mul(mul(dmu, dT[c], e), du[a][c] + du[c][a], e);
      }
      vis[a] = mul(mu, lap + (1.0 / 3.0) * ddiv, e) + mul(muv, ddiv, e) + cross +
               mul(mul(dmuv - (2.0 / 3.0) * dmu, dT[a], e), div, e);
    }
  }

  // y-direction inviscid terms, replaced at the non-reflective boundaries
  DN Yp, Yv;
  bool dropc = false;
  if (j == 0 || j == P.ny - 1) {
    unsigned char fl = P.bcflags[(j == P.ny - 1 ? (long long)P.nx * P.nz : 0) + (long long)k * P.nx + i];
    DN c = dsqrt(P.gamma * mul(p, rcp(rho, e), e), e);
    DN rc = mul(rho, c, e);
    DN rcv = mul(rc, du[Y][Y], e);
    DN Xp = 0.5 * mul(u[Y] + c, dp[Y] + rcv, e);
    DN Xm = 0.5 * mul(u[Y] - c, dp[Y] - rcv, e);
    if (fl & 1) Xp = dn(0.0, 0.0);
    if (fl & 2) Xm = dn(0.0, 0.0);
    dropc = (fl & 4) != 0;
    Yp = -(Xp + Xm);
    Yv = -mul(Xp - Xm, rcp(rc, e), e);
  } else {
    Yp = -(mul(u[Y], dp[Y], e) + P.gamma * mul(p, du[Y][Y], e));
    Yv = -(mul(u[Y], du[Y][Y], e) + mul(dp[Y], rcp(rho, e), e));
  }
  DN src = heat + Phi;
  DN pt_ = Yp;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (a != Y) pt_ = pt_ - (mul(u[a], dp[a], e) + P.gamma * mul(p, du[a][a], e));
  pt_ = pt_ + (P.gamma - 1.0) * src;
  res[0] = pt_.w;
  DN irho = rcp(rho, e);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    DN r = dn(0.0, 0.0);
    if (c == Y) {
      r = Yv;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != Y) r = r - mul(u[a], du[c][a], e);
    } else {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a == Y && dropc) continue;
        r = r - mul(u[a], du[c][a], e);
      }
      r = r - mul(dp[c], irho, e);
    }
    r = r + mul(vis[c], irho, e);
    res[1 + c] = r.w;
  }
  DN st = dn(0.0, 0.0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == Y && dropc) continue;
    st = st - mul(u[a], ds[a], e);
  }
  st = st + mul(P.R * rcp(p, e), src, e);
  res[D + 1] = st.w;
}

template <int D>
__global__ void __launch_bounds__(128) k_point(const PointParams P) {
  const double e = *P.eps;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)gridDim.x * blockDim.x) {
    int i = (int)(pt % P.nx);
    int j = (int)((pt / P.nx) % P.ny);
    int k = (int)(pt / ((long long)P.nx * P.ny));
    double r0[D + 2], r1[D + 2];
    point_rhs<D>(P, pt, i, j, k, 0, e, r0);
    point_rhs<D>(P, pt, i, j, k, 1, e, r1);
#pragma unroll
    for (int a = 0; a < D + 2; ++a) {
      long long o = (long long)a * P.npts + pt;
      double2 vv = P.v[o];
      // out = J v - shift v
      double2 r = make_double2(r0[a] - (P.shift.x * vv.x - P.shift.y * vv.y), r1[a] - (P.shift.x * vv.y + P.shift.y * vv.x));
      P.out[o] = r;
    }
  }
}

// base state as complex fields + base temperature (imaginary parts zero)
__global__ void k_base_fields(const double* q0, long long npts, int nv, double pref, double igam, double icp, double R,
                              double2* bv, double2* bT) {
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < npts; pt += (long long)gridDim.x * blockDim.x) {
    for (int a = 0; a < nv; ++a) bv[(long long)a * npts + pt] = make_double2(q0[(long long)a * npts + pt], 0.0);
    double p = q0[pt], s = q0[(long long)(nv - 1) * npts + pt];
    double rho = pow(p / pref, igam) * exp(-s * icp);
    bT[pt] = make_double2(p / (rho * R), 0.0);
  }
}

struct PackParams {
  const double* q0;
  const double2* scratch;
  double* btab;
  long long npts, nbase;
  int nx, ny, D, homog, visc;
  int s_Tw, s_d1[3][6], s_d2[3][4], s_mix[3][3];
  const double* eta_y;
  const double* eta_yy;
  double pref, igam, icp, R;
};

__global__ void k_pack_base(const PackParams P) {
  const int D = P.D;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < P.nbase; b += (long long)gridDim.x * blockDim.x) {
    long long pt = P.homog ? b * P.nx : b;
    int j = (int)((pt / P.nx) % P.ny);
    double ey = P.eta_y[j], eyy = P.eta_yy[j];
    auto out = [&](int slot, double v) { P.btab[(long long)slot * P.nbase + b] = v; };
    auto S_ = [&](int slot) { return P.scratch[(long long)slot * P.npts + pt].x; };
    for (int f = 0; f < D + 2; ++f) out(bt_val(D, f), P.q0[(long long)f * P.npts + pt]);
    double p = P.q0[pt], s = P.q0[(long long)(D + 1) * P.npts + pt];
    double rho = pow(p / P.pref, P.igam) * exp(-s * P.icp);
    out(bt_val(D, D + 2), p / (rho * P.R));
    out(bt_val(D, D + 3), rho);
    for (int ax = 0; ax < D; ++ax) {
      for (int f = 0; f < D + 3; ++f) {
        double v = 0.0;
        if (P.s_d1[ax][f] >= 0) v = S_(P.s_d1[ax][f]) * (ax == 1 ? ey : 1.0);
        out(bt_d1(D, ax, f), v);
      }
      for (int g = 0; g < D + 1; ++g) {
        double v = 0.0;
        if (P.s_d2[ax][g] >= 0) {
          v = S_(P.s_d2[ax][g]);
          if (ax == 1) {
            int f = g < D ? 1 + g : D + 2;
            v = v * ey * ey + S_(P.s_d1[1][f]) * eyy;
          }
        }
        out(bt_d2(D, ax, g), v);
      }
      for (int c = 0; c < D; ++c) {
        double v = 0.0;
        if (ax != c && P.s_mix[ax][c] >= 0) v = S_(P.s_mix[ax][c]) * ((ax == 1 || c == 1) ? ey : 1.0);
        out(bt_mix(D, ax, c), v);
      }
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static void fill_axis_tables(AxisTables& A, std::vector<double>& host) {
  const int n = A.n;
  host.assign((size_t)6 * n, 0.0);
  for (int kind = 0; kind < 2; ++kind) {
    double* l = host.data() + (size_t)kind * 3 * n;
    double* dinv = l + n;
    double* m = l + 2 * n;
    const double al = kind == 0 ? 1.0 / 3.0 : 2.0 / 11.0;
    const double r = (-1.0 + std::sqrt(1.0 - 4.0 * al * al)) / (2.0 * al);
    A.K[kind] = (int)std::ceil(56.0 * std::log(2.0) / -std::log(std::fabs(r))) + 1;
    if (A.periodic) {
      const double c = -al / r;  // circulant = c (1 - r S^-1)(1 - r S)
      for (int t = 0; t < n; ++t) { l[t] = -r; dinv[t] = 1.0 / c; m[t] = -r; }
    } else {
      std::vector<double> a(n, al), b(n, 1.0), cc(n, al);
      if (kind == 0) { cc[0] = 2.0; a[n - 1] = 2.0; a[1] = cc[1] = a[n - 2] = cc[n - 2] = 0.25; }
      else { cc[0] = 11.0; a[n - 1] = 11.0; a[1] = cc[1] = a[n - 2] = cc[n - 2] = 0.1; }
      a[0] = 0.0;
      cc[n - 1] = 0.0;
      double d = b[0];
      l[0] = 0.0;
      dinv[0] = 1.0 / d;
      m[0] = cc[0] / d;
      for (int t = 1; t < n; ++t) {
        l[t] = a[t] / d;
        d = b[t] - l[t] * cc[t - 1];
        dinv[t] = 1.0 / d;
        m[t] = cc[t] / d;
      }
    }
  }
}

static void make_slots(StabHandle* h) {
  Slots& S = h->slots;
  const int D = h->dim;
  int c = 0;
  S.Tw = c++;
  for (int ax = 0; ax < 3; ++ax) {
    for (int f = 0; f < 6; ++f) S.d1[ax][f] = -1;
    for (int g = 0; g < 4; ++g) S.d2[ax][g] = -1;
    for (int k = 0; k < 3; ++k) S.mix[ax][k] = -1;
  }
  for (int ax = 0; ax < D; ++ax) {
    for (int f = 0; f < D + 3; ++f)
      if (f < D + 2 || h->visc) S.d1[ax][f] = c++;
    if (h->visc)
      for (int g = 0; g < D + 1; ++g) S.d2[ax][g] = c++;
  }
  if (h->visc)
    for (int i = 0; i < D; ++i)
      for (int k = 0; k < D; ++k)
        if (i != k) S.mix[i][k] = c++;
  S.count = c;
}

static cudaError_t run_pass(StabHandle* h, int axis, const PassParams& base_params, const std::vector<LineJob>& jobs) {
  if (jobs.empty()) return cudaSuccess;
  PassParams P = base_params;
  const AxisTables& A = h->ax[axis];
  P.axis = axis;
  P.n = A.n;
  P.nx = h->nx;
  P.ny = h->ny;
  P.periodic = A.periodic;
  P.h = A.h;
  P.tab[0] = A.tab[0];
  P.tab[1] = A.tab[1];
  P.K[0] = A.K[0];
  P.K[1] = A.K[1];
  P.stride = axis == 0 ? 1 : axis == 1 ? h->nx : (long long)h->nx * h->ny;
  P.nlines = h->npts / A.n;
  // interior weights: first (a/2h, b/4h), second (a/h^2, b/4h^2)
  P.c1[0] = (14.0 / 9.0) / (2.0 * A.h);
  P.c2[0] = (1.0 / 9.0) / (4.0 * A.h);
  P.c1[1] = (12.0 / 11.0) / (A.h * A.h);
  P.c2[1] = (3.0 / 11.0) / (4.0 * A.h * A.h);
  const int n = A.n;
  int L = (int)(98304 / (3 * 16 * (long long)n));
  if (L > 32) L = 32;
  if (L < 1) L = 1;
  P.L = L;
  P.C = 64;
  P.nchunks = (n + P.C - 1) / P.C;
  int threads = 2 * L * P.nchunks;
  threads = ((threads + 31) / 32) * 32;
  size_t smem = (size_t)3 * n * L * sizeof(double2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;  // lines longer than 4266 points
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_line_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  for (size_t j0 = 0; j0 < jobs.size(); j0 += STAB_MAX_JOBS) {
    P.njobs = (int)std::min<size_t>(STAB_MAX_JOBS, jobs.size() - j0);
    for (int q = 0; q < P.njobs; ++q) P.job[q] = jobs[j0 + q];
    dim3 grid((unsigned)((P.nlines + L - 1) / L), (unsigned)P.njobs);
    k_line_pass<<<grid, threads, smem, h->stream>>>(P);
  }
  return cudaGetLastError();
}

// all derivative passes for field sources src[f] (f = 0..D+2)
static cudaError_t run_derivatives(StabHandle* h, const double2* const* src) {
  const int D = h->dim;
  const Slots& S = h->slots;
  double2* sc = h->d_scratch;
  auto slot = [&](int s) -> double2* { return s >= 0 ? sc + (long long)s * h->npts : nullptr; };
  PassParams P{};
  const int nf = h->visc ? D + 3 : D + 2;
  auto field_jobs = [&](int ax, std::vector<LineJob>& jobs) {
    for (int f = 0; f < nf; ++f) {
      LineJob J;
      J.in = src[f];
      J.out1 = slot(S.d1[ax][f]);
      J.out2 = nullptr;
      if (h->visc) {
        if (f >= 1 && f <= D) J.out2 = slot(S.d2[ax][f - 1]);
        if (f == D + 2) J.out2 = slot(S.d2[ax][D]);
      }
      jobs.push_back(J);
    }
  };
  cudaError_t err;
  {  // y
    std::vector<LineJob> jobs;
    field_jobs(1, jobs);
    if ((err = run_pass(h, 1, P, jobs)) != cudaSuccess) return err;
  }
  if (D == 3) {  // z, plus d/dz of d/dy v and d/dy w
    std::vector<LineJob> jobs;
    field_jobs(2, jobs);
    if (h->visc) {
      jobs.push_back(LineJob{slot(S.d1[1][2]), slot(S.mix[2][1]), nullptr});
      jobs.push_back(LineJob{slot(S.d1[1][3]), slot(S.mix[1][2]), nullptr});
    }
    if ((err = run_pass(h, 2, P, jobs)) != cudaSuccess) return err;
  }
  {  // x, plus d/dx of d/dy u, d/dy v (and d/dz u, d/dz w)
    std::vector<LineJob> jobs;
    field_jobs(0, jobs);
    if (h->visc) {
      jobs.push_back(LineJob{slot(S.d1[1][2]), slot(S.mix[0][1]), nullptr});
      jobs.push_back(LineJob{slot(S.d1[1][1]), slot(S.mix[1][0]), nullptr});
      if (D == 3) {
        jobs.push_back(LineJob{slot(S.d1[2][3]), slot(S.mix[0][2]), nullptr});
        jobs.push_back(LineJob{slot(S.d1[2][1]), slot(S.mix[2][0]), nullptr});
      }
    }
    if ((err = run_pass(h, 0, P, jobs)) != cudaSuccess) return err;
  }
  return cudaSuccess;
}

static PointParams point_params(StabHandle* h, const double2* v) {
  PointParams P{};
  P.v = v;
  P.scratch = h->d_scratch;
  P.npts = h->npts;
  P.nx = h->nx;
  P.ny = h->ny;
  P.nz = h->nz;
  P.D = h->dim;
  P.homog = h->homog;
  P.visc = h->visc;
  P.s_Tw = h->slots.Tw;
  for (int a = 0; a < 3; ++a) {
    for (int f = 0; f < 6; ++f) P.s_d1[a][f] = h->slots.d1[a][f];
    for (int g = 0; g < 4; ++g) P.s_d2[a][g] = h->slots.d2[a][g];
    for (int c = 0; c < 3; ++c) P.s_mix[a][c] = h->slots.mix[a][c];
  }
  P.btab = h->d_btab;
  P.nbase = h->nbase;
  P.eta_y = h->d_metric;
  P.eta_yy = h->d_metric + h->ny;
  P.bcflags = h->d_bcflags;
  P.eps = h->d_eps;
  P.gamma = h->gamma;
  P.R = h->R;
  P.cp = h->cp;
  P.Pr = h->Pr;
  P.S = h->S;
  P.Re = h->Re;
  P.bulk = h->bulk;
  P.C.ig = 1.0 / h->gamma;
  P.C.omig = 1.0 - 1.0 / h->gamma;
  P.C.icp = 1.0 / h->cp;
  return P;
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_norm2(StabHandle* h, const double2* v, long long n, double* d_out, int mode) {
  k_norm2_partial<<<h->red_blocks, 256, 0, h->stream>>>(v, n, h->d_red);
  k_norm2_final<<<1, 32, 0, h->stream>>>(h->d_red, h->red_blocks, d_out, mode, h->q0norm, h->opts.eps);
  return cudaGetLastError();
}

cudaError_t jv_setup(StabHandle* h, const double* q0_host) {
  const int D = h->dim;
  cudaError_t err;
  make_slots(h);
  // axis tables: x (0) periodic, y (1) bounded in eta, z (2) periodic
  const int lens[3] = {h->nx, h->ny, h->nz};
  for (int ax = 0; ax < 3; ++ax) {
    AxisTables& A = h->ax[ax];
    A.n = lens[ax];
    A.periodic = ax != 1;
    A.h = ax == 0 ? h->lx / h->nx : ax == 1 ? 1.0 / (h->ny - 1) : (D == 3 ? h->lz / h->nz : 1.0);
    A.tab[0] = A.tab[1] = nullptr;
    if (ax >= D) continue;
    std::vector<double> host;
    fill_axis_tables(A, host);
    double* d;
    if ((err = cudaMalloc(&d, host.size() * sizeof(double))) != cudaSuccess) return err;
    cudaMemcpy(d, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice);
    A.tab[0] = d;
    A.tab[1] = d + 3 * A.n;
  }
  // metric eta_y = 1/y', eta_yy = -y''/y'^3
  {
    std::vector<double> met(2 * (size_t)h->ny);
    for (int j = 0; j < h->ny; ++j) {
      double eta = (double)j / (h->ny - 1), yp, ypp;
      if (h->stretch == 0.0) { yp = h->ly1 - h->ly0; ypp = 0.0; }
      else {
        double be = h->stretch, half = 0.5 * (h->ly1 - h->ly0), sb = std::sinh(be);
        yp = half * 2.0 * be * std::cosh(be * (2.0 * eta - 1.0)) / sb;
        ypp = half * 4.0 * be * be * std::sinh(be * (2.0 * eta - 1.0)) / sb;
      }
      met[j] = 1.0 / yp;
      met[h->ny + j] = -ypp / (yp * yp * yp);
    }
    if ((err = cudaMalloc(&h->d_metric, met.size() * sizeof(double))) != cudaSuccess) return err;
    cudaMemcpy(h->d_metric, met.data(), met.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  // non-reflective boundary flags from the base state (frozen switch)
  {
    const long long nxz = (long long)h->nx * h->nz;
    std::vector<unsigned char> fl(2 * nxz, 0);
    const double pref = h->R, Y = 1;
    (void)Y;
    for (int top = 0; top < 2; ++top)
      for (int k = 0; k < h->nz; ++k)
        for (int i = 0; i < h->nx; ++i) {
          int j = top ? h->ny - 1 : 0;
          long long pt = ((long long)k * h->ny + j) * h->nx + i;
          double p0 = q0_host[pt], v0 = q0_host[2 * h->npts + pt], s0 = q0_host[(long long)(D + 1) * h->npts + pt];
          double rho0 = std::pow(p0 / pref, 1.0 / h->gamma) * std::exp(-s0 / h->cp);
          double c0 = std::sqrt(h->gamma * p0 / rho0);
          bool in_plus = top ? (v0 + c0 < 0.0) : (v0 + c0 > 0.0);
          bool in_minus = top ? (v0 - c0 < 0.0) : (v0 - c0 > 0.0);
          bool dropc = top ? (v0 < 0.0) : (v0 > 0.0);
          fl[top * nxz + (long long)k * h->nx + i] = (in_plus ? 1 : 0) | (in_minus ? 2 : 0) | (dropc ? 4 : 0);
        }
    if ((err = cudaMalloc(&h->d_bcflags, fl.size())) != cudaSuccess) return err;
    cudaMemcpy(h->d_bcflags, fl.data(), fl.size(), cudaMemcpyHostToDevice);
  }
  // scratch, reductions, eps
  if ((err = cudaMalloc(&h->d_scratch, (size_t)h->slots.count * h->npts * sizeof(double2))) != cudaSuccess) return err;
  h->red_blocks = 1024;
  if ((err = cudaMalloc(&h->d_red, (h->red_blocks + 64) * sizeof(double))) != cudaSuccess) return err;
  h->d_eps = h->d_red + h->red_blocks;
  k_set_scalar<<<1, 1, 0, h->stream>>>(h->d_eps, 0.0);
  // base tables: derivatives of the base fields through the same passes
  const int nbt = bt_count(D);
  if ((err = cudaMalloc(&h->d_btab, (size_t)nbt * h->nbase * sizeof(double))) != cudaSuccess) return err;
  double2* bv;
  if ((err = cudaMalloc(&bv, (size_t)(h->nv + 1) * h->npts * sizeof(double2))) != cudaSuccess) return err;
  double2* bT = bv + (long long)h->nv * h->npts;
  int thr = 256;
  k_base_fields<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(h->d_q0, h->npts, h->nv, h->R, 1.0 / h->gamma,
                                                                1.0 / h->cp, h->R, bv, bT);
  const double2* src[6];
  for (int f = 0; f < D + 2; ++f) src[f] = bv + (long long)f * h->npts;
  src[D + 2] = bT;
  if ((err = run_derivatives(h, src)) != cudaSuccess) return err;
  PackParams K{};
  K.q0 = h->d_q0;
  K.scratch = h->d_scratch;
  K.btab = h->d_btab;
  K.npts = h->npts;
  K.nbase = h->nbase;
  K.nx = h->nx;
  K.ny = h->ny;
  K.D = D;
  K.homog = h->homog;
  K.visc = h->visc;
  K.s_Tw = h->slots.Tw;
  for (int a = 0; a < 3; ++a) {
    for (int f = 0; f < 6; ++f) K.s_d1[a][f] = h->slots.d1[a][f];
    for (int g = 0; g < 4; ++g) K.s_d2[a][g] = h->slots.d2[a][g];
    for (int c = 0; c < 3; ++c) K.s_mix[a][c] = h->slots.mix[a][c];
  }
  K.eta_y = h->d_metric;
  K.eta_yy = h->d_metric + h->ny;
  K.pref = h->R;
  K.igam = 1.0 / h->gamma;
  K.icp = 1.0 / h->cp;
  K.R = h->R;
  k_pack_base<<<grid_for(h->nbase, thr), thr, 0, h->stream>>>(K);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if ((err = cudaStreamSynchronize(h->stream)) != cudaSuccess) return err;
  cudaFree(bv);
  return cudaSuccess;
}

cudaError_t jv_apply(StabHandle* h, const double2* v, double2* out, double2 shift, int eps_mode) {
  cudaError_t err;
  if (eps_mode == 2) {
    if (h->last_eps_mode != 2) k_set_scalar<<<1, 1, 0, h->stream>>>(h->d_eps, 0.0);
  } else {
    if ((err = launch_norm2(h, v, h->n, h->d_eps, 2)) != cudaSuccess) return err;
  }
  h->last_eps_mode = eps_mode;
  PointParams P = point_params(h, v);
  P.out = out;
  P.shift = shift;
  double2* Tw = h->d_scratch + (long long)h->slots.Tw * h->npts;
  const int thr = 128;
  if (h->visc) k_temperature<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P, Tw);
  const int D = h->dim;
  const double2* src[6];
  for (int f = 0; f < D + 2; ++f) src[f] = v + (long long)f * h->npts;
  src[D + 2] = Tw;
  if ((err = run_derivatives(h, src)) != cudaSuccess) return err;
  if (D == 2) k_point<2><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P);
  else k_point<3><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P);
  h->stats.jv_calls++;
  return cudaGetLastError();
}
