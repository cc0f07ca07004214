// Pointwise part of the right-hand side N(q) (Eq. navier_stokes), evaluated
// on scaled differences: given the base state a (from tables) and the scaled
// perturbation w = (q - q0)/eps of every value and derivative at one point,
// returns [N(q0 + eps w) - N(q0)]/eps at that point, free of cancellation.
// eps = 0 gives the exact tangent.  Shared by the J v kernel and by the
// block-Jacobi assembly (which feeds it unit perturbations).
#pragma once
#include "internal.cuh"

namespace pw {

// ---------------------------------------------------------------------------
// Difference numbers: a = base value, w = (perturbed - base)/eps.
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

// Below, x is the relative perturbation e w / a.  For |x| < 1e-4 each
// function is its Taylor series about 0 up to x^4 (the truncation error is
// below 1e-20 relative); otherwise the closed form.
// 1/(1+x)
__device__ __forceinline__ double inv1p(double x) {
  if (fabs(x) < 1e-4) return fma(x, fma(x, fma(x, x - 1.0, 1.0), -1.0), 1.0);
  return 1.0 / (1.0 + x);
}
// (sqrt(1+x) - 1)/x, binomial series 1/2 - x/8 + x^2/16 - 5x^3/128 + 7x^4/256
__device__ __forceinline__ double sqrt1p_m1_over(double x) {
  if (fabs(x) < 1e-4) return fma(x, fma(x, fma(x, fma(x, 7.0 / 256.0, -5.0 / 128.0), 1.0 / 16.0), -1.0 / 8.0), 0.5);
  return (sqrt(1.0 + x) - 1.0) / x;
}
// (e^z - 1)/z = 1 + z/2 + z^2/6 + z^3/24 + z^4/120
__device__ __forceinline__ double expm1_over(double z) {
  if (fabs(z) < 1e-4) return fma(z, fma(z, fma(z, fma(z, 1.0 / 120.0, 1.0 / 24.0), 1.0 / 6.0), 0.5), 1.0);
  return expm1(z) / z;
}
// ln(1+z)/z = 1 - z/2 + z^2/3 - z^3/4 + z^4/5
__device__ __forceinline__ double log1p_over(double z) {
  if (fabs(z) < 1e-4) return fma(z, fma(z, fma(z, fma(z, 0.2, -0.25), 1.0 / 3.0), -0.5), 1.0);
  return log1p(z) / z;
}

// 1/x with the base reciprocal from a table:  w = -w_x / (a (a + e w_x))
__device__ __forceinline__ DN rcp_t(DN x, double inva, double e) {
  return dn(inva, -x.w * inva * inva * inv1p(e * x.w * inva));
}
// sqrt(x) with sqrt(a) and 1/a from tables:  w = w_x g(e w_x / a) / sqrt(a)
__device__ __forceinline__ DN sqrt_t(DN x, double sqa, double inva, double e) {
  return dn(sqa, x.w * (sqa * inva) * sqrt1p_m1_over(e * x.w * inva));
}

// ---------------------------------------------------------------------------
// Three-part difference numbers in FP32: w1 = first-order (tangent) part,
// w2 = the rest of the scaled difference.  Used to evaluate only the O(eps)
// remainder [N(q0 + eps w) - N(q0)]/eps - J w, whose size relative to J w is
// eps |w| / |a|; FP32 rounding of that remainder is far below the 1e-10
// target.  Inputs carry w2 = 0.
// ---------------------------------------------------------------------------
struct DN3 {
  float a, w1, w2;
};
__device__ __forceinline__ DN3 dn3(float a, float w1, float w2) { return DN3{a, w1, w2}; }
__device__ __forceinline__ DN3 operator+(DN3 x, DN3 y) { return dn3(x.a + y.a, x.w1 + y.w1, x.w2 + y.w2); }
__device__ __forceinline__ DN3 operator-(DN3 x, DN3 y) { return dn3(x.a - y.a, x.w1 - y.w1, x.w2 - y.w2); }
__device__ __forceinline__ DN3 operator-(DN3 x) { return dn3(-x.a, -x.w1, -x.w2); }
__device__ __forceinline__ DN3 operator*(double c, DN3 x) {
  float cf = (float)c;
  return dn3(cf * x.a, cf * x.w1, cf * x.w2);
}
__device__ __forceinline__ DN3 add(DN3 x, double c) { return dn3(x.a + (float)c, x.w1, x.w2); }
__device__ __forceinline__ DN3 mul(DN3 x, DN3 y, double ed) {
  const float e = (float)ed;
  float w1 = fmaf(x.a, y.w1, x.w1 * y.a);
  float w2 = fmaf(x.a, y.w2, fmaf(x.w2, y.a, e * (x.w1 + x.w2) * (y.w1 + y.w2)));
  return dn3(x.a * y.a, w1, w2);
}
// x/(1+x) and (1/(1+x) - 1) = -x/(1+x)
__device__ __forceinline__ float xinv1pf(float x) {
  if (fabsf(x) < 1e-3f) return x * fmaf(x, fmaf(x, 1.0f - x, -1.0f), 1.0f);
  return x / (1.0f + x);
}
__device__ __forceinline__ DN3 rcp_t(DN3 x, double inva_d, double ed) {
  const float inva = (float)inva_d, i2 = inva * inva;
  const float w = x.w1 + x.w2;
  const float X = (float)ed * w * inva;
  return dn3(inva, -x.w1 * i2, fmaf(-x.w2, i2, w * i2 * xinv1pf(X)));
}
// (sqrt(1+x) - 1)/x - 1/2 = x (-1/8 + x/16 - 5x^2/128 + ...)
__device__ __forceinline__ float sqrt_corr(float x) {
  if (fabsf(x) < 1e-3f) return x * fmaf(x, fmaf(x, -5.0f / 128.0f, 1.0f / 16.0f), -1.0f / 8.0f);
  return (sqrtf(1.0f + x) - 1.0f) / x - 0.5f;
}
__device__ __forceinline__ DN3 sqrt_t(DN3 x, double sqa_d, double inva_d, double ed) {
  const float sqa = (float)sqa_d, inva = (float)inva_d, k = sqa * inva;
  const float w = x.w1 + x.w2;
  const float X = (float)ed * w * inva;
  return dn3(sqa, 0.5f * k * x.w1, fmaf(0.5f * k, x.w2, w * k * sqrt_corr(X)));
}

// ---------------------------------------------------------------------------
// Closure: rho(p, s) = (p/p_ref)^{1/gamma} e^{-s/c_p}, T = (p/p_ref)^{(gamma-1)/gamma} e^{s/c_p}
//   rho(q0 + e w)/rho0 = exp(x_rho),  x_rho = (1/gamma) ln(1 + e wp/p0) - e ws/c_p
// ---------------------------------------------------------------------------
struct ClosureK {
  double ig, omig, icp;  // 1/gamma, 1 - 1/gamma, 1/c_p
};
__device__ __forceinline__ double closure_lq(double wp, double ip0, double e) {
  double q = wp * ip0;
  return q * log1p_over(e * q);
}
__device__ __forceinline__ double closure_rho_w(const ClosureK& C, double rho0, double lq, double ws, double e) {
  double x = fma(C.ig, lq, -ws * C.icp);
  return rho0 * expm1_over(e * x) * x;
}
__device__ __forceinline__ double closure_T_w(const ClosureK& C, double T0, double lq, double ws, double e) {
  double x = fma(C.omig, lq, ws * C.icp);
  return T0 * expm1_over(e * x) * x;
}

// e^z - 1 - z over z, and ln(1+z) - z over z, for the FP32 remainder
__device__ __forceinline__ float expm1_m1_over_f(float z) {
  if (fabsf(z) < 1e-3f) return z * fmaf(z, fmaf(z, 1.0f / 24.0f, 1.0f / 6.0f), 0.5f);
  return expm1f(z) / z - 1.0f;
}
__device__ __forceinline__ float log1p_m1_over_f(float z) {
  if (fabsf(z) < 1e-3f) return z * fmaf(z, fmaf(z, -0.25f, 1.0f / 3.0f), -0.5f);
  return log1pf(z) / z - 1.0f;
}

// Closure functions by number type: rho from the inputs (p, s).
__device__ __forceinline__ DN make_rho(const ClosureK& C, double rho0, double ip0, DN p, DN s, double e) {
  return dn(rho0, closure_rho_w(C, rho0, closure_lq(p.w, ip0, e), s.w, e));
}
__device__ __forceinline__ DN3 make_rho(const ClosureK& C, double rho0, double ip0, DN3 p, DN3 s, double ed) {
  const float e = (float)ed, r0 = (float)rho0;
  const float q = p.w1 * (float)ip0;
  const float X1 = fmaf((float)C.ig, q, -s.w1 * (float)C.icp);
  const float X2 = (float)C.ig * q * log1p_m1_over_f(e * q);
  const float X = X1 + X2;
  return dn3(r0, r0 * X1, r0 * fmaf(X, expm1_m1_over_f(e * X), X2));
}

// ---------------------------------------------------------------------------
// Base tables: real arrays of length nbase (physical derivatives).
// ---------------------------------------------------------------------------
enum Extra { X_IRHO = 0, X_IP, X_IT, X_SQT, X_ITS, X_C, X_RC, X_IRC, X_COUNT };
__host__ __device__ __forceinline__ int bt_val(int D, int f) { (void)D; return f; }  // p,u..,s,T,rho
__host__ __device__ __forceinline__ int bt_d1(int D, int ax, int f) { return (D + 4) + ax * (D + 3) + f; }
__host__ __device__ __forceinline__ int bt_d2(int D, int ax, int g) { return (D + 4) + D * (D + 3) + ax * (D + 1) + g; }
__host__ __device__ __forceinline__ int bt_mix(int D, int i, int k) {
  return (D + 4) + D * (D + 3) + D * (D + 1) + i * D + k;
}
__host__ __device__ __forceinline__ int bt_extra(int D, int x) {
  return (D + 4) + D * (D + 3) + D * (D + 1) + D * D + x;
}
__host__ __device__ __forceinline__ int bt_count(int D) { return bt_extra(D, X_COUNT); }

struct Phys {
  double gamma, R, cp, Pr, S, Re, bulk;
  ClosureK C;
  int visc;
};

// Scaled perturbation at one point for one real direction.  Fields f:
// 0 = p, 1..D = u_i, D+1 = s, D+2 = T; d2 fields g: 0..D-1 = u_i, D = T.
template <int D, class V = double>
struct WIn {
  V v[D + 3];
  V d1[D][D + 3];
  V d2[D][D + 1];
  V mix[D][D];  // d/dx_i d/dx_k u_k, i != k
};

__device__ __forceinline__ DN mk(double a, double w) { return dn(a, w); }
__device__ __forceinline__ DN3 mk3(double a, float w) { return dn3((float)a, w, 0.0f); }
template <class Num>
struct NumOps;
template <>
struct NumOps<DN> {
  typedef double V;
  __device__ static DN make(double a, double w) { return dn(a, w); }
  __device__ static DN zero() { return dn(0.0, 0.0); }
};
template <>
struct NumOps<DN3> {
  typedef float V;
  __device__ static DN3 make(double a, float w) { return dn3((float)a, w, 0.0f); }
  __device__ static DN3 zero() { return dn3(0.0f, 0.0f, 0.0f); }
};

// out[0..D+1] = scaled differences of the (p, u_i, s) tendencies as numbers
// of type Num (DN: FP64 full difference; DN3: FP32 with the first-order part
// split off).  B(slot) reads the base table entry at this point.  bcfl:
// non-reflective flags of a y-boundary row (bit0 drop X+, bit1 drop X-,
// bit2 drop y-convection), bc_row: the point lies on one.
template <int D, class Num, class BaseFn>
__device__ __forceinline__ void rhs_num(const Phys& P, const BaseFn& B, const WIn<D, typename NumOps<Num>::V>& W,
                                        double e, bool bc_row, unsigned bcfl, Num* out) {
  typedef NumOps<Num> O;
  const int Y = 1;
  Num p = O::make(B(bt_val(D, 0)), W.v[0]);
  Num u[D];
#pragma unroll
  for (int a = 0; a < D; ++a) u[a] = O::make(B(bt_val(D, 1 + a)), W.v[1 + a]);
  Num s = O::make(B(bt_val(D, D + 1)), W.v[D + 1]);
  const auto rho0 = B(bt_val(D, D + 3)), irho0 = B(bt_extra(D, X_IRHO)), ip0 = B(bt_extra(D, X_IP));
  Num rho = make_rho(P.C, rho0, ip0, p, s, e);
  Num irho = rcp_t(rho, irho0, e);
  Num dp[D], ds[D], du[D][D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    dp[a] = O::make(B(bt_d1(D, a, 0)), W.d1[a][0]);
    ds[a] = O::make(B(bt_d1(D, a, D + 1)), W.d1[a][D + 1]);
#pragma unroll
    for (int c = 0; c < D; ++c) du[c][a] = O::make(B(bt_d1(D, a, 1 + c)), W.d1[a][1 + c]);
  }
  Num div = du[0][0];
#pragma unroll
  for (int a = 1; a < D; ++a) div = div + du[a][a];

  Num src = O::zero();
  Num vis[D];
#pragma unroll
  for (int a = 0; a < D; ++a) vis[a] = O::zero();
  if (P.visc) {
    const auto T0 = B(bt_val(D, D + 2)), iT0 = B(bt_extra(D, X_IT));
    Num T = O::make(T0, W.v[D + 2]);
    Num dT[D];
#pragma unroll
    for (int a = 0; a < D; ++a) dT[a] = O::make(B(bt_d1(D, a, D + 2)), W.d1[a][D + 2]);
    // Sutherland: mu = (1+S)/Re T^{3/2}/(T+S);  dmu/dT = mu (3/(2T) - 1/(T+S))
    Num sqT = sqrt_t(T, B(bt_extra(D, X_SQT)), iT0, e);
    const auto iTS0 = B(bt_extra(D, X_ITS));
    Num rTS = rcp_t(add(T, P.S), iTS0, e);
    Num mu = ((1.0 + P.S) / P.Re) * mul(mul(T, sqT, e), rTS, e);
    Num dmu = mul(mu, 1.5 * rcp_t(T, iT0, e) - rTS, e);
    const double kl = P.cp / P.Pr;
    Num lapT = O::zero(), gT2 = O::zero();
#pragma unroll
    for (int a = 0; a < D; ++a) {
      lapT = lapT + O::make(B(bt_d2(D, a, D)), W.d2[a][D]);
      gT2 = gT2 + mul(dT[a], dT[a], e);
    }
    Num heat = kl * (mul(mu, lapT, e) + mul(dmu, gT2, e));
    Num SS = O::zero();
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        Num sij = 0.5 * (du[a][c] + du[c][a]);
        SS = SS + mul(sij, sij, e);
      }
    Num div2 = mul(div, div, e);
    Num Phi = 2.0 * mul(mu, SS - (1.0 / 3.0) * div2, e) + P.bulk * mul(mu, div2, e);
    src = heat + Phi;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      Num lap = O::zero(), ddiv = O::zero(), cross = O::zero();
#pragma unroll
      for (int c = 0; c < D; ++c) {
        Num d2ac = O::make(B(bt_d2(D, c, a)), W.d2[c][a]);  // d^2 u_a / dx_c^2
        lap = lap + d2ac;
        ddiv = ddiv + (c == a ? d2ac : O::make(B(bt_mix(D, a, c)), W.mix[a][c]));
        cross = cross + mul(dT[c], du[a][c] + du[c][a], e);
      }
      vis[a] = mul(mu, lap + (1.0 / 3.0) * ddiv, e) + P.bulk * mul(mu, ddiv, e) + mul(dmu, cross, e) +
               mul(mul((P.bulk - 2.0 / 3.0) * dmu, dT[a], e), div, e);
    }
  }

  // y-direction inviscid terms, replaced at the non-reflective boundaries
  Num Yp, Yv;
  bool dropc = false;
  if (bc_row) {
    Num c = sqrt_t(P.gamma * mul(p, irho, e), B(bt_extra(D, X_C)), rho0 * ip0 / P.gamma, e);
    Num rc = mul(rho, c, e);
    Num rcv = mul(rc, du[Y][Y], e);
    Num Xp = 0.5 * mul(u[Y] + c, dp[Y] + rcv, e);
    Num Xm = 0.5 * mul(u[Y] - c, dp[Y] - rcv, e);
    if (bcfl & 1) Xp = O::zero();
    if (bcfl & 2) Xm = O::zero();
    dropc = (bcfl & 4) != 0;
    Yp = -(Xp + Xm);
    Yv = -mul(Xp - Xm, rcp_t(rc, B(bt_extra(D, X_IRC)), e), e);
  } else {
    Yp = -(mul(u[Y], dp[Y], e) + P.gamma * mul(p, du[Y][Y], e));
    Yv = -(mul(u[Y], du[Y][Y], e) + mul(dp[Y], irho, e));
  }
  Num pt = Yp;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (a != Y) pt = pt - (mul(u[a], dp[a], e) + P.gamma * mul(p, du[a][a], e));
  pt = pt + (P.gamma - 1.0) * src;
  out[0] = pt;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    Num r;
    if (c == Y) {
      r = Yv;
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != Y) r = r - mul(u[a], du[c][a], e);
    } else {
      r = O::zero();
#pragma unroll
      for (int a = 0; a < D; ++a) {
        if (a == Y && dropc) continue;
        r = r - mul(u[a], du[c][a], e);
      }
      r = r - mul(dp[c], irho, e);
    }
    r = r + mul(vis[c], irho, e);
    out[1 + c] = r;
  }
  Num st = O::zero();
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == Y && dropc) continue;
    st = st - mul(u[a], ds[a], e);
  }
  st = st + mul(P.R * rcp_t(p, ip0, e), src, e);
  out[D + 1] = st;
}


// res = scaled difference in FP64 (full evaluation)
template <int D, class BaseFn>
__device__ __forceinline__ void rhs_diff(const Phys& P, const BaseFn& B, const WIn<D>& W, double e, bool bc_row,
                                         unsigned bcfl, double* res) {
  DN o[D + 2];
  rhs_num<D, DN>(P, B, W, e, bc_row, bcfl, o);
#pragma unroll
  for (int a = 0; a < D + 2; ++a) res[a] = o[a].w;
}

// Number of linear inputs of the pointwise map: v (D+2), T, d1, d2, mixed.
__host__ __device__ constexpr int nw_inputs(int D) { return (D + 3) + D * (D + 3) + D * (D + 1) + D * D; }

}  // namespace pw
