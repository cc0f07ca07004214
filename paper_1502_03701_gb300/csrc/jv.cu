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
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <map>
#include <mutex>

#include "internal.cuh"

#include "pairs.cuh"
#include "pointwise.cuh"

using pw::bt_count;
using pw::bt_d1;
using pw::bt_d2;
using pw::bt_extra;
using pw::bt_mix;
using pw::bt_val;

namespace {

// ---------------------------------------------------------------------------
// Line pass: compact derivatives along one axis for a batch of fields.
// A CTA stages L lines x n points of one field in shared memory; each thread
// runs one chunk of one line for one derivative kind, first forward (with a
// warm-up of K points, after which the influence of the unknown start value
// has decayed below 2^-56), then backward.
// ---------------------------------------------------------------------------
// Division by an invariant divisor with a multiply and a shift (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// p = 31 + ceil(log2 d), m = ceil(2^p / d), x / d = umulhi(x, m) >> (p - 32)
// for 0 <= x < 2^31.
struct FastDiv {
  unsigned d, m;
  int s;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{d, 0u, 0};
  if (d > 1) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    const int p = 31 + l;
    f.m = (unsigned)(((1ull << p) + d - 1) / d);
    f.s = p - 32;
  }
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv& f) {
  return f.d == 1 ? x : (__umulhi(x, f.m) >> f.s);
}

struct PassParams {
  LineJob job[STAB_MAX_JOBS];
  int njobs;
  int axis, n, nx, ny;
  long long nlines;
  long long stride;
  int L, C, nchunks;
  int KP;  // 1: kinds in turn, 2: side by side, 3: in turn with the input reloaded (2 planes)
  int LS;
  FastDiv divn, divL, divnx;  // division by n, L and nx  // padded shared-memory line stride in doubles, n + n/32 + 1
  int periodic;
  double c1[2], c2[2];  // interior stencil weights per kind
  float c1h[2], c1l[2], c2h[2], c2l[2];  // the same weights as FP32 pairs (ff = 1)
  int ff;  // 1: interior right-hand sides in FP32 pair arithmetic on exponent-shifted inputs
  double h;
  const double* tab[2];
  const float* tabf[2];  // FP32 copies [l'(n), m(n)] for the far part of the warm-up
  int K[2];
  int Wn[2];             // near part of the warm-up kept in FP64
  const int* gate;  // when set and nonzero the launch does nothing (graph-captured GMRES after convergence)
};

__device__ __forceinline__ long long line_base(const PassParams& P, long long l) {
  if (P.axis == 0) return l * P.nx;
  if (P.axis == 1) {  // l < 2^31 (grids have fewer than 2^31 points)
    const long long q = fdiv((unsigned)l, P.divnx);
    return q * (long long)P.nx * P.ny + (l - q * P.nx);
  }
  return l;
}

// t mod n for t within a few periods of [0, n) (no integer division)
__device__ __forceinline__ int wrap_small(int t, int n) {
  while (t < 0) t += n;
  while (t >= n) t -= n;
  return t;
}

// shared-memory index of line point t: one pad double after every 32-point
// chunk so that the chunk starts fall in different banks
__device__ __forceinline__ int sidx(int t) { return t + (t >> 5); }

// right-hand side of the one-sided and Pade closure rows of a bounded line
// (t < 2 or t > n - 3) from the values f(q)
template <class Get>
__device__ __forceinline__ double closure_rhs(const PassParams& P, Get f, int t, int kind) {
  const int n = P.n;
  const double h = P.h;
  if (kind == 0) {
    if (t == 0) return (-2.5 * f(0) + 2.0 * f(1) + 0.5 * f(2)) / h;
    if (t == n - 1) return (2.5 * f(n - 1) - 2.0 * f(n - 2) - 0.5 * f(n - 3)) / h;
    return 0.75 * (f(t + 1) - f(t - 1)) / h;
  }
  const double ih2 = 1.0 / (h * h);
  if (t == 0) return (13.0 * f(0) - 27.0 * f(1) + 15.0 * f(2) - f(3)) * ih2;
  if (t == n - 1) return (13.0 * f(n - 1) - 27.0 * f(n - 2) + 15.0 * f(n - 3) - f(n - 4)) * ih2;
  return 1.2 * (f(t + 1) - 2.0 * f(t) + f(t - 1)) * ih2;
}

// neighbour indices t-2 .. t+2 (wrapped on periodic lines)
__device__ __forceinline__ void stencil_idx(const PassParams& P, int t, int& tm2, int& tm1, int& tp1, int& tp2) {
  tm2 = t - 2; tm1 = t - 1; tp1 = t + 1; tp2 = t + 2;
  if (P.periodic) {
    const int n = P.n;
    tm2 = wrap_small(tm2, n); tm1 = wrap_small(tm1, n); tp1 = wrap_small(tp1, n); tp2 = wrap_small(tp2, n);
  }
}

// interior right-hand side from the five values f_{t-2} .. f_{t+2} (f_t is
// only read by the second derivative)
__device__ __forceinline__ double interior_rhs(const PassParams& P, int kind, double fm2, double fm1, double f0,
                                               double fp1, double fp2) {
  if (kind == 0) return fma(P.c1[0], fp1 - fm1, P.c2[0] * (fp2 - fm2));
  return fma(P.c1[1], fp1 - 2.0 * f0 + fm1, P.c2[1] * (fp2 - 2.0 * f0 + fm2));
}

// right-hand side (B f)_t of the compact scheme for one real component
__device__ __forceinline__ double stencil_rhs(const PassParams& P, const double* fl, int t, int kind) {
  auto f = [&](int q) { return fl[sidx(q)]; };
  if (!P.periodic && (t < 2 || t > P.n - 3)) return closure_rhs(P, f, t, kind);
  int tm2, tm1, tp1, tp2;
  stencil_idx(P, t, tm2, tm1, tp1, tp2);
  return interior_rhs(P, kind, f(tm2), f(tm1), kind ? f(t) : 0.0, f(tp1), f(tp2));
}

// interior right-hand side in pair arithmetic (values f * 2^-sh)
__device__ __forceinline__ ffn interior_rhs_ff(const PassParams& P, int kind, ffn fm2, ffn fm1, ffn f0, ffn fp1,
                                               ffn fp2) {
  const ffn c1{P.c1h[kind], P.c1l[kind]}, c2{P.c2h[kind], P.c2l[kind]};
  if (kind == 0) return ff_add(ff_prod(c1, ff_sub(fp1, fm1)), ff_prod(c2, ff_sub(fp2, fm2)));
  const ffn m2{-2.0f * f0.hi, -2.0f * f0.lo};
  return ff_add(ff_prod(c1, ff_add(ff_add(fp1, fm1), m2)), ff_prod(c2, ff_add(ff_add(fp2, fm2), m2)));
}

// The same right-hand side from a line of FP32 pairs holding f * 2^-sh: the
// interior rows in pair arithmetic (~2^-47 relative; no FP64 work but the
// final recombination), the closure rows in FP64 on the recombined values.
__device__ __forceinline__ double stencil_rhs_ff(const PassParams& P, const float2* fl, int t, int kind, int sh) {
  auto f = [&](int q) { const float2 v = fl[sidx(q)]; return ffn{v.x, v.y}; };
  if (!P.periodic && (t < 2 || t > P.n - 3)) {
    auto fd = [&](int q) { return ff_to_d_scaled(f(q), sh); };
    return closure_rhs(P, fd, t, kind);
  }
  int tm2, tm1, tp1, tp2;
  stencil_idx(P, t, tm2, tm1, tp1, tp2);
  return ff_to_d_scaled(interior_rhs_ff(P, kind, f(tm2), f(tm1), kind ? f(t) : ffn{0.0f, 0.0f}, f(tp1), f(tp2)), sh);
}

// biased exponent of |d| (0 for zero and subnormals)
__device__ __forceinline__ int dexp(double d) { return (int)((__double_as_longlong(d) >> 52) & 0x7FF); }

constexpr long long kLineSmemMax = 200 * 1024;  // dynamic shared memory opt-in of k_line_pass
constexpr long long kLineSmemExtra = 16;        // after the planes: the CTA's input exponent (pair stencil)

// FP32 value of a double with integer operations (the FP64 pipe is the
// bottleneck here): the high part of ff_split.
__device__ __forceinline__ float d2f_hi(double d) { return ff_split(d).hi; }

// Shared memory (doubles): F[comp][lt][LS] (the input lines) and
// W[kind][comp][lt][LS] (right-hand side, then forward-sweep values, in
// place); LS = padded line stride.  P.KP derivative kinds are done at once
// (2: first and second side by side, more threads; 1: one after the other
// with half the shared memory).  Per kind:
//   1. W = right-hand side of the compact scheme, scaled by the pivots'
//      reciprocals (stencil weights on periodic axes, 1/d_t on bounded);
//   2. carry-in of each chunk's forward sweep: the recurrence over the K
//      points before the chunk (read-only; far part in FP32, whose error is
//      damped below 2^-56 by the near part of length Wn);
//   3. forward sweep of the own chunk, in place (W becomes g');
//   4. carry-in of the back substitution over the K points after the chunk;
//   5. back substitution of the own chunk, written to global memory.
// Threads: (kind, comp, line, chunk); x lines: chunk fastest, strided lines:
// line fastest (neighbouring lines are neighbouring addresses).
// Steps 2-5 for one kind on the plane Wk of this thread's line and component
// (block-uniform call: contains barriers).
__device__ __forceinline__ void line_sweeps(const PassParams& P, double* Wk, int kind, bool act, int t0, int t1,
                                            long long base, int comp, double2* out) {
  const int n = P.n;
  const double* tl = P.tab[kind & 1];
  const double* tm = tl + 2 * n;
  const float* tlf = P.tabf[kind & 1];
  const float* tmf = tlf + n;
  const int K = P.K[kind & 1], Wn = P.Wn[kind & 1];
  // 2. forward carry-in g'_{t0-1}
  double g = 0.0;
  if (act) {
    if (P.periodic) {
      const double lv = __ldg(tl);
      const float lvf = __ldg(tlf);
      float gf = 0.0f;
      int tt = wrap_small(t0 - K, n);
      int s = t0 - K;
      for (; s < t0 - Wn; ++s) {
        gf = fmaf(-lvf, gf, d2f_hi(Wk[sidx(tt)]));
        if (++tt == n) tt = 0;
      }
      g = f2d_exact(gf);
      for (; s < t0; ++s) {
        g = fma(-lv, g, Wk[sidx(tt)]);
        if (++tt == n) tt = 0;
      }
    } else if (t0 > 0) {
      const int ts = (t0 - K < 8) ? 0 : t0 - K;
      const int tw = max(ts, t0 - Wn);
      float gf = 0.0f;
      for (int t = ts; t < tw; ++t) gf = fmaf(-__ldg(tlf + t), gf, d2f_hi(Wk[sidx(t)]));
      g = f2d_exact(gf);
      for (int t = tw; t < t0; ++t) g = fma(-__ldg(tl + t), g, Wk[sidx(t)]);
    }
  }
  __syncthreads();
  // 3. forward sweep of the own chunk, in place
  if (act) {
    if (P.periodic) {
      const double lv = __ldg(tl);
      for (int t = t0; t < t1; ++t) {
        g = fma(-lv, g, Wk[sidx(t)]);
        Wk[sidx(t)] = g;
      }
    } else {
      for (int t = t0; t < t1; ++t) {
        g = fma(-__ldg(tl + t), g, Wk[sidx(t)]);
        Wk[sidx(t)] = g;
      }
    }
  }
  __syncthreads();
  // 4. back-substitution carry-in x_{t1}, 5. own chunk
  if (act) {
    double x = 0.0;
    double* o = (double*)out + comp;
    if (P.periodic) {
      const double mm = __ldg(tm);
      const float mmf = __ldg(tmf);
      const int te = t1 - 1 + K;
      int tt = wrap_small(te, n);
      int s = te;
      float xf = 0.0f;
      for (; s > t1 - 1 + Wn; --s) {
        xf = fmaf(-mmf, xf, d2f_hi(Wk[sidx(tt)]));
        if (--tt < 0) tt = n - 1;
      }
      x = f2d_exact(xf);
      for (; s >= t1; --s) {
        x = fma(-mm, x, Wk[sidx(tt)]);
        if (--tt < 0) tt = n - 1;
      }
      for (int t = t1 - 1; t >= t0; --t) {
        x = fma(-mm, x, Wk[sidx(t)]);
        o[2 * (base + (long long)t * P.stride)] = x;
      }
    } else {
      if (t1 < n) {
        const int te = (t1 - 1 + K > n - 9) ? n - 1 : t1 - 1 + K;
        const int tw = min(te, t1 - 1 + Wn);
        float xf = 0.0f;
        for (int t = te; t > tw; --t) xf = fmaf(-__ldg(tmf + t), xf, d2f_hi(Wk[sidx(t)]));
        x = f2d_exact(xf);
        for (int t = tw; t >= t1; --t) x = fma(-__ldg(tm + t), x, Wk[sidx(t)]);
      }
      for (int t = t1 - 1; t >= t0; --t) {
        x = fma(-__ldg(tm + t), x, Wk[sidx(t)]);
        o[2 * (base + (long long)t * P.stride)] = x;
      }
    }
  }
}

// One CTA's work of the line pass: line block bx of job by.
template <bool FF>
__device__ __forceinline__ void line_pass_body(const PassParams& P, const unsigned bx, const unsigned by) {
  if (P.gate && *P.gate) return;
  extern __shared__ double sm[];
  const LineJob J = P.job[by];
  const int n = P.n, L = P.L, KP = P.KP;
  const int LS = P.LS;
  const size_t plane = (size_t)L * LS;
  double* F = sm;              // 2 planes
  double* W = sm + 2 * plane;  // 2 KP planes
  int* sE = (int*)(sm + (size_t)(2 + 2 * KP) * plane);  // FF: largest input exponent of the CTA
  const long long l0 = (long long)bx * L;
  if (FF) {
    if (threadIdx.x == 0) *sE = 0;
    __syncthreads();
  }
  int em = 0;
  auto load_lines = [&]() {
    for (int idx = threadIdx.x; idx < n * L; idx += blockDim.x) {
      int lt, t;
      if (P.axis == 0) { lt = (int)fdiv(idx, P.divn); t = idx - lt * n; } else { t = (int)fdiv(idx, P.divL); lt = idx - t * L; }
      const long long l = l0 + lt;
      double2 val = make_double2(0.0, 0.0);
      if (l < P.nlines) val = J.in[line_base(P, l) + (long long)t * P.stride];
      F[(size_t)lt * LS + sidx(t)] = val.x;
      F[plane + (size_t)lt * LS + sidx(t)] = val.y;
      if (FF) em = max(em, max(dexp(val.x), dexp(val.y)));
    }
  };
  const int per = L * P.nchunks;
  const int ch = P.axis == 0 ? threadIdx.x % P.nchunks : (threadIdx.x / L) % P.nchunks;
  const int lt = P.axis == 0 ? (threadIdx.x / P.nchunks) % L : threadIdx.x % L;
  const int comp = (threadIdx.x / per) & 1;
  const int t0 = ch * P.C, t1 = min(n, t0 + P.C);
  const int nk = J.out2 ? 2 : 1;
  load_lines();
  int sh = 0;
  if (FF) {
    // exact power-of-two scaling into the FP32 exponent range, then the
    // split of every staged value into a pair, in place
    em = __reduce_max_sync(0xffffffffu, em);
    if ((threadIdx.x & 31) == 0) atomicMax(sE, em);
    __syncthreads();
    sh = *sE - 1023;
    for (int idx = threadIdx.x; idx < 2 * n * L; idx += blockDim.x) {
      const int r2 = (int)fdiv(idx, P.divn);
      const int t = idx - r2 * n;
      double* p = F + (size_t)r2 * LS + sidx(t);  // r2 = c * L + line: planes are L * LS apart
      const ffn v = ff_split_scaled(*p, sh);
      *(float2*)p = make_float2(v.hi, v.lo);
    }
  }
  const int kt = threadIdx.x / (2 * per);  // this thread's kind within a group of KP
  const bool active = kt < KP && (l0 + lt) < P.nlines;
  const long long base = active ? line_base(P, l0 + lt) : 0;
  for (int kb = 0; kb < nk; kb += KP) {
    const int kg = min(KP, nk - kb);  // kinds in this group
    __syncthreads();  // F complete / the previous group's W no longer read
    for (int idx = threadIdx.x; idx < kg * 2 * L * n; idx += blockDim.x) {
      const int rest = (int)fdiv(idx, P.divn);
      const int t = idx - rest * n;
      const int r2 = (int)fdiv(rest, P.divL);
      const int l = rest - r2 * L, c = r2 & 1, k = r2 >> 1;
      const size_t off = (size_t)c * plane + (size_t)l * LS;
      double r = FF ? stencil_rhs_ff(P, (const float2*)(F + off), t, kb + k, sh) : stencil_rhs(P, F + off, t, kb + k);
      if (!P.periodic) r *= __ldg(P.tab[kb + k] + n + t);  // bounded: row scale 1/d_t (periodic: in c1, c2)
      W[(size_t)(k * 2 + c) * plane + (size_t)l * LS + sidx(t)] = r;
    }
    __syncthreads();
    const int kind = kb + kt;
    double* Wk = W + (size_t)((kt & 1) * 2 + comp) * plane + (size_t)lt * LS;
    line_sweeps(P, Wk, kind, active && kt < kg, t0, t1, base, comp, kind == 0 ? J.out1 : J.out2);
  }
}

template <bool FF>
__global__ void k_line_pass(const PassParams P) {
  line_pass_body<FF>(P, blockIdx.x, blockIdx.y);
}

// Compact variant (KP = 3): kinds in turn, the input reloaded per kind into
// the only plane of each component, half the shared memory of the
// kinds-in-turn layout.  Each thread turns its own chunk of input into
// right-hand sides in place, left to right, with the five stencil values in
// registers: the two values on each side of the chunk (which neighbouring
// threads overwrite) and the closure rows of a bounded line are taken before
// a barrier.  The arithmetic is that of the other layouts, so the results
// are the same.
constexpr int kCompactMaxThreads = 512;

// the value (input of one component) at line index q of this thread's chunk
// [t0, t1) or of its halo (two points on each side, read before the barrier)
template <class V>
struct Window {
  V m2, m1, p0, p1;  // f(t0 - 2), f(t0 - 1), f(t1), f(t1 + 1)
};

template <bool FF>
__device__ __forceinline__ void line_pass_compact_body(const PassParams& P, const unsigned bx, const unsigned by) {
  if (P.gate && *P.gate) return;
  extern __shared__ double sm[];
  const LineJob J = P.job[by];
  const int n = P.n, L = P.L;
  const int LS = P.LS;
  const size_t plane = (size_t)L * LS;
  int* sE = (int*)(sm + 2 * plane);  // FF: largest input exponent of the CTA
  const long long l0 = (long long)bx * L;
  const int per = L * P.nchunks;
  const int ch = P.axis == 0 ? threadIdx.x % P.nchunks : (threadIdx.x / L) % P.nchunks;
  const int lt = P.axis == 0 ? (threadIdx.x / P.nchunks) % L : threadIdx.x % L;
  const int comp = (threadIdx.x / per) & 1;
  const int t0 = ch * P.C, t1 = min(n, t0 + P.C);
  const int nk = J.out2 ? 2 : 1;
  const bool active = threadIdx.x < 2 * per && (l0 + lt) < P.nlines;
  const long long base = active ? line_base(P, l0 + lt) : 0;
  double* Wc = sm + (size_t)comp * plane + (size_t)lt * LS;
  using V = typename std::conditional<FF, ffn, double>::type;
  auto at = [&](int q) -> V {  // staged value at line index q (wrapped on periodic lines)
    if (P.periodic) q = wrap_small(q, n);
    if constexpr (FF) {
      const float2 v = ((const float2*)Wc)[sidx(q)];
      return ffn{v.x, v.y};
    } else {
      return Wc[sidx(q)];
    }
  };
  if (FF && threadIdx.x == 0) *sE = 0;
  int sh = 0;
  for (int kind = 0; kind < nk; ++kind) {
    __syncthreads();  // the previous kind's sweeps no longer read the planes
    int em = 0;
    for (int idx = threadIdx.x; idx < n * L; idx += blockDim.x) {
      int l, t;
      if (P.axis == 0) { l = (int)fdiv(idx, P.divn); t = idx - l * n; } else { t = (int)fdiv(idx, P.divL); l = idx - t * L; }
      double2 val = make_double2(0.0, 0.0);
      if (l0 + l < P.nlines) val = J.in[line_base(P, l0 + l) + (long long)t * P.stride];
      sm[(size_t)l * LS + sidx(t)] = val.x;
      sm[plane + (size_t)l * LS + sidx(t)] = val.y;
      if (FF) em = max(em, max(dexp(val.x), dexp(val.y)));
    }
    if (FF) {
      if (kind == 0) {
        em = __reduce_max_sync(0xffffffffu, em);
        if ((threadIdx.x & 31) == 0) atomicMax(sE, em);
      }
      __syncthreads();
      sh = *sE - 1023;
      for (int idx = threadIdx.x; idx < 2 * n * L; idx += blockDim.x) {
        const int r2 = (int)fdiv(idx, P.divn);
        const int t = idx - r2 * n;
        double* p = sm + (size_t)r2 * LS + sidx(t);
        const ffn v = ff_split_scaled(*p, sh);
        *(float2*)p = make_float2(v.hi, v.lo);
      }
    }
    __syncthreads();
    // halo values and the closure rows of this chunk, before any overwrite
    Window<V> w{};
    double cl[4] = {0.0, 0.0, 0.0, 0.0};  // rows 0, 1, n - 2, n - 1 (bounded lines)
    const bool bounded = !P.periodic;
    if (active) {
      if (P.periodic || t0 >= 2) w.m2 = at(t0 - 2);
      if (P.periodic || t0 >= 1) w.m1 = at(t0 - 1);
      if (P.periodic || t1 < n) w.p0 = at(t1);
      if (P.periodic || t1 + 1 < n) w.p1 = at(t1 + 1);
      if (bounded) {
        const int rows[4] = {0, 1, n - 2, n - 1};
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (rows[k] >= t0 && rows[k] < t1) {
            double r;
            if constexpr (FF) {
              auto fd = [&](int q) { return ff_to_d_scaled(at(q), sh); };
              r = closure_rhs(P, fd, rows[k], kind);
            } else {
              auto fd = [&](int q) { return at(q); };
              r = closure_rhs(P, fd, rows[k], kind);
            }
            cl[k] = r * __ldg(P.tab[kind] + n + rows[k]);
          }
      }
    }
    __syncthreads();
    if (active) {
      // value at q for q in [t0 - 2, t1 + 2): own chunk from shared memory
      // (positions >= the current row are not yet overwritten), else the halo
      auto get = [&](int q) -> V {
        if (q >= t0 && q < t1) return at(q);
        return q == t0 - 2 ? w.m2 : q == t0 - 1 ? w.m1 : q == t1 ? w.p0 : w.p1;
      };
      V fm2 = w.m2, fm1 = w.m1, f0 = get(t0), fp1 = get(t0 + 1), fp2 = get(t0 + 2);
      for (int t = t0; t < t1; ++t) {
        double r;
        if (bounded && (t < 2 || t > n - 3)) {
          r = t == 0 ? cl[0] : t == 1 ? cl[1] : t == n - 2 ? cl[2] : cl[3];
        } else {
          if constexpr (FF) r = ff_to_d_scaled(interior_rhs_ff(P, kind, fm2, fm1, f0, fp1, fp2), sh);
          else r = interior_rhs(P, kind, fm2, fm1, f0, fp1, fp2);
          if (bounded) r *= __ldg(P.tab[kind] + n + t);
        }
        const V next = (t + 3 < t1 + 2) ? get(t + 3) : fp2;  // f(t + 3) for the next row
        Wc[sidx(t)] = r;
        fm2 = fm1;
        fm1 = f0;
        f0 = fp1;
        fp1 = fp2;
        fp2 = next;
      }
    }
    __syncthreads();
    line_sweeps(P, Wc, kind, active, t0, t1, base, comp, kind == 0 ? J.out1 : J.out2);
  }
}

template <bool FF>
__global__ void __launch_bounds__(kCompactMaxThreads) k_line_pass_compact(const PassParams P) {
  line_pass_compact_body<FF>(P, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Reductions: ||v||^2 in a fixed order (deterministic), then epsilon.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double block_sum(double s, double* red) {
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  return t;  // valid in thread 0
}

// mode 0: out = sum;  mode 1: out = sqrt(sum);  mode 2: epsilon from ||v||
__device__ __forceinline__ double norm_result(double s, int mode, double q0norm, double fixed_eps) {
  if (mode == 0) return s;
  if (mode == 1) return sqrt(s);
  if (fixed_eps > 0.0) return fixed_eps;
  return s > 0.0 ? 1.4901161193847656e-08 * (1.0 + q0norm) / sqrt(s) : 0.0;  // sqrt(2^-52)
}

// ||v||^2 in one launch: per-block sums, then the last block to finish adds
// them in block order (fixed order, reproducible) and resets the counter.
// Block bidx of nb blocks.
__device__ __forceinline__ void norm2_body(const double2* __restrict__ v, long long n, double* partial, unsigned* counter,
                                           double* out, int mode, double q0norm, double fixed_eps, unsigned bidx,
                                           unsigned nb) {
  __shared__ double red[32];
  __shared__ bool last;
  double s = 0.0;
  for (long long i = (long long)bidx * blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) {
    double2 z = v[i];
    s = fma(z.x, z.x, fma(z.y, z.y, s));
  }
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) {
    partial[bidx] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double a = 0.0;
  for (int b = threadIdx.x; b < (int)nb; b += blockDim.x) a += ((volatile double*)partial)[b];
  __syncthreads();
  const double tot = block_sum(a, red);
  if (threadIdx.x == 0) {
    *out = norm_result(tot, mode, q0norm, fixed_eps);
    *counter = 0u;
  }
}

__global__ void k_norm2(const double2* __restrict__ v, long long n, double* partial, unsigned* counter, double* out,
                        int mode, double q0norm, double fixed_eps, const int* gate) {
  if (gate && *gate) return;
  norm2_body(v, n, partial, counter, out, mode, q0norm, fixed_eps, blockIdx.x, gridDim.x);
}

__global__ void k_norm2_partial(const double2* __restrict__ v, long long n, double* partial, const int* gate) {
  if (gate && *gate) return;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 z = v[i];
    s = fma(z.x, z.x, fma(z.y, z.y, s));
  }
  __shared__ double red[32];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_norm2_final(const double* partial, int nb, double* out, int mode, double q0norm, double fixed_eps,
                              const int* gate) {
  if (gate && *gate) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += partial[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = norm_result(s, mode, q0norm, fixed_eps);
}

__global__ void k_set_scalar(double* p, double v) { *p = v; }

// ---------------------------------------------------------------------------
// Pointwise kernels
// ---------------------------------------------------------------------------
struct PointParams {
  const double2* v;
  const double2* scratch;
  long long npts;
  int nx, ny, nz;
  int homog;
  int s_Tw;
  int s_d1[3][6], s_d2[3][4], s_mix[3][3];
  const double* btab;
  long long nbase;
  const double* eta_y;
  const double* eta_yy;
  const double* eta_y_f;   // same values (read into FP32 by the remainder path)
  const double* eta_yy_f;
  const unsigned char* bcflags;
  const double* eps;
  double2* out;
  double2 shift;
  pw::Phys phys;
  const int* gate;  // as PassParams::gate
  FastDiv divnx, divny;  // division by nx and ny (points < 2^31)
};

// y index of grid point pt ([z][y][x] order)
__device__ __forceinline__ int row_of(const PointParams& P, long long pt) {
  const unsigned r = fdiv((unsigned)pt, P.divnx);
  return (int)(r - fdiv(r, P.divny) * P.ny);
}

__global__ void k_temperature(const PointParams P, double2* Tw) {
  if (P.gate && *P.gate) return;
  const int D = P.nz > 1 ? 3 : 2;
  const double e = *P.eps;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)gridDim.x * blockDim.x) {
    int j = row_of(P, pt);
    long long b = P.homog ? j : pt;
    double ip0 = P.btab[bt_extra(D, pw::X_IP) * P.nbase + b];
    double T0 = P.btab[bt_val(D, D + 2) * P.nbase + b];
    double2 wp = P.v[pt], ws = P.v[(long long)(D + 1) * P.npts + pt];
    double t0 = pw::closure_T_w(P.phys.C, T0, pw::closure_lq(wp.x, ip0, e), ws.x, e);
    double t1 = pw::closure_T_w(P.phys.C, T0, pw::closure_lq(wp.y, ip0, e), ws.y, e);
    Tw[pt] = make_double2(t0, t1);
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_point(const PointParams P) {
  if (P.gate && *P.gate) return;
  const double e = *P.eps;
  const bool visc = P.phys.visc;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(pt % P.nx);
    const int j = row_of(P, pt);
    const int k = (int)(pt / ((long long)P.nx * P.ny));
    const long long b = P.homog ? j : pt;
    const double ey = P.eta_y[j], eyy = P.eta_yy[j];
    const bool bc_row = (j == 0 || j == P.ny - 1);
    const unsigned fl = bc_row ? P.bcflags[(j == P.ny - 1 ? (long long)P.nx * P.nz : 0) + (long long)k * P.nx + i] : 0u;
    auto B = [&](int slot) { return P.btab[(long long)slot * P.nbase + b]; };
    auto S = [&](int slot) { return P.scratch[(long long)slot * P.npts + pt]; };
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      auto pick = [&](double2 z) { return part ? z.y : z.x; };
      pw::WIn<D> W;
#pragma unroll
      for (int f = 0; f < D + 2; ++f) W.v[f] = pick(P.v[(long long)f * P.npts + pt]);
      W.v[D + 2] = visc ? pick(S(P.s_Tw)) : 0.0;
#pragma unroll
      for (int ax = 0; ax < D; ++ax) {
        const double sc = ax == 1 ? ey : 1.0;
#pragma unroll
        for (int f = 0; f < D + 3; ++f) W.d1[ax][f] = (f < D + 2 || visc) ? pick(S(P.s_d1[ax][f])) * sc : 0.0;
      }
      if (visc) {
#pragma unroll
        for (int ax = 0; ax < D; ++ax)
#pragma unroll
          for (int g = 0; g < D + 1; ++g) {
            double w = pick(S(P.s_d2[ax][g]));
            if (ax == 1) w = fma(w, ey * ey, pick(S(P.s_d1[1][g < D ? 1 + g : D + 2])) * eyy);
            W.d2[ax][g] = w;
          }
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c)
            W.mix[a][c] = a == c ? 0.0 : pick(S(P.s_mix[a][c])) * ((a == 1 || c == 1) ? ey : 1.0);
      }
      double res[D + 2];
      pw::rhs_diff<D>(P.phys, B, W, e, bc_row, fl, res);
#pragma unroll
      for (int a = 0; a < D + 2; ++a) {
        const long long o = (long long)a * P.npts + pt;
        double2 vv = P.v[o];
        double sv = part ? (P.shift.x * vv.y + P.shift.y * vv.x) : (P.shift.x * vv.x - P.shift.y * vv.y);
        double r = res[a] - sv;
        if (part) P.out[o].y = r; else P.out[o].x = r;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fast pointwise path for a base state that depends on y only.  The map from
// the scaled perturbation inputs (values and derivatives at a point) to the
// tendencies is, to first order, linear with coefficients that depend on the
// row only: C_j (D+2 x NW), tabulated once by feeding unit inputs through the
// FP64 tangent.  J v at a point is then C_j w in FP64; for eps > 0 the
// remaining O(eps) part of the quotient is added, evaluated in FP32.
// ---------------------------------------------------------------------------
template <int D, class V>
__device__ __forceinline__ void set_input(pw::WIn<D, V>& W, int idx, V val) {
  if (idx < D + 3) { W.v[idx] = val; return; }
  idx -= D + 3;
  if (idx < D * (D + 3)) { W.d1[idx / (D + 3)][idx % (D + 3)] = val; return; }
  idx -= D * (D + 3);
  if (idx < D * (D + 1)) { W.d2[idx / (D + 1)][idx % (D + 1)] = val; return; }
  idx -= D * (D + 1);
  W.mix[idx / D][idx % D] = val;
}

template <int D>
__global__ void k_coeffs(const PointParams P, double* coef) {
  constexpr int NW = pw::nw_inputs(D);
  const int j = blockIdx.x, k = threadIdx.x;
  if (k >= NW) return;
  pw::WIn<D> W;
#pragma unroll
  for (int q = 0; q < NW; ++q) set_input<D, double>(W, q, q == k ? 1.0 : 0.0);
  auto B = [&](int slot) { return P.btab[(long long)slot * P.nbase + j]; };
  const bool bc_row = (j == 0 || j == P.ny - 1);
  const unsigned fl = bc_row ? P.bcflags[(j == P.ny - 1 ? (long long)P.nx * P.nz : 0)] : 0u;
  double res[D + 2];
  pw::rhs_diff<D>(P.phys, B, W, 0.0, bc_row, fl, res);
  for (int a = 0; a < D + 2; ++a) coef[((long long)j * (D + 2) + a) * NW + k] = res[a];
}



// Inputs: raw line-pass outputs (eta-derivatives in y); the coefficients have
// the y metric folded in (k_coeffs_fold) and are stored as FP32 pairs.  The
// tangent part C_j w is formed with exact FP32 two-products of the pairs and
// two-sum accumulation (~2^-47 relative per term), the O(eps) remainder in
// FP32 from the inputs' high parts and FP32 base tables: no FP64 products.
template <int D>
__device__ __forceinline__ void point_fast_body(const PointParams& P, const ffn* __restrict__ coefp,
                                                const float* __restrict__ btab_f, unsigned bidx, unsigned nb) {
  constexpr int NW = pw::nw_inputs(D);
  constexpr int o2 = (D + 3) + D * (D + 3), om = o2 + D * (D + 1);
  const double e = *P.eps;
  const bool visc = P.phys.visc;
  for (long long pt = (long long)bidx * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)nb * blockDim.x) {
    const int j = row_of(P, pt);
    const bool bc_row = (j == 0 || j == P.ny - 1);
    const unsigned fl = bc_row ? P.bcflags[(j == P.ny - 1 ? (long long)P.nx * P.nz : 0)] : 0u;
    const float2* Cp = (const float2*)(coefp + (long long)j * (D + 2) * NW);
    auto S = [&](int slot) { return P.scratch[(long long)slot * P.npts + pt]; };
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
      auto pick = [&](double2 z) { return part ? z.y : z.x; };
      double w[NW];
#pragma unroll
      for (int f = 0; f < D + 2; ++f) w[f] = pick(P.v[(long long)f * P.npts + pt]);
      w[D + 2] = visc ? pick(S(P.s_Tw)) : 0.0;
#pragma unroll
      for (int ax = 0; ax < D; ++ax)
#pragma unroll
        for (int f = 0; f < D + 3; ++f) w[D + 3 + ax * (D + 3) + f] = (f < D + 2 || visc) ? pick(S(P.s_d1[ax][f])) : 0.0;
#pragma unroll
      for (int ax = 0; ax < D; ++ax)
#pragma unroll
        for (int g = 0; g < D + 1; ++g) w[o2 + ax * (D + 1) + g] = visc ? pick(S(P.s_d2[ax][g])) : 0.0;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int c = 0; c < D; ++c) w[om + a * D + c] = (visc && a != c) ? pick(S(P.s_mix[a][c])) : 0.0;
      ffn wp[NW];
#pragma unroll
      for (int q = 0; q < NW; ++q) wp[q] = ff_split(w[q]);
      double res[D + 2];
#pragma unroll
      for (int a = 0; a < D + 2; ++a) {
        ffn acc{0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < NW; ++q) {
          const float2 c = __ldg(Cp + a * NW + q);
          ff_acc_prod(acc, ffn{c.x, c.y}, wp[q]);
        }
        res[a] = ff_to_d(acc);
      }
      if (e != 0.0) {  // O(eps) remainder of the quotient, FP32, physical (metric-applied) inputs
        const float ey = ff_split(P.eta_y[j]).hi, eyy = ff_split(P.eta_yy[j]).hi;
        pw::WIn<D, float> Wf;
#pragma unroll
        for (int q = 0; q < NW; ++q) set_input<D, float>(Wf, q, wp[q].hi);
#pragma unroll
        for (int f = 0; f < D + 3; ++f) Wf.d1[1][f] *= ey;
#pragma unroll
        for (int g = 0; g < D + 1; ++g)
          Wf.d2[1][g] = fmaf(Wf.d2[1][g], ey * ey, wp[D + 3 + (D + 3) + (g < D ? 1 + g : D + 2)].hi * eyy);
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
          for (int c = 0; c < D; ++c)
            if (a == 1 || c == 1) Wf.mix[a][c] *= ey;
        auto Bf = [&](int slot) { return btab_f[(long long)slot * P.nbase + j]; };
        pw::DN3 o[D + 2];
        pw::rhs_num<D, pw::DN3>(P.phys, Bf, Wf, e, bc_row, fl, o);
#pragma unroll
        for (int a = 0; a < D + 2; ++a) res[a] += f2d_exact(o[a].w2);
      }
#pragma unroll
      for (int a = 0; a < D + 2; ++a) {
        const long long o = (long long)a * P.npts + pt;
        double2 vv = P.v[o];
        double sv = part ? (P.shift.x * vv.y + P.shift.y * vv.x) : (P.shift.x * vv.x - P.shift.y * vv.y);
        double r = res[a] - sv;
        if (part) P.out[o].y = r; else P.out[o].x = r;
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(128, D == 2 ? 4 : 3) k_point_fast(const PointParams P, const ffn* __restrict__ coefp,
                                                   const float* __restrict__ btab_f) {
  if (P.gate && *P.gate) return;
  point_fast_body<D>(P, coefp, btab_f, blockIdx.x, gridDim.x);
}

// Fold the y metric into the per-row coefficients so that the pointwise kernel
// can use the line passes' eta-derivatives directly:
//   f_y = f_eta ey,  f_yy = f_etaeta ey^2 + f_eta eyy,  mixed with y: x ey.
template <int D>
__global__ void k_coeffs_fold(const double* coef, const double* eta_y, const double* eta_yy, int ny, double* out) {
  constexpr int NW = pw::nw_inputs(D);
  constexpr int o1 = D + 3, o2 = (D + 3) + D * (D + 3), om = o2 + D * (D + 1);
  const int j = blockIdx.x, a = threadIdx.x;
  if (j >= ny || a >= D + 2) return;
  const double ey = eta_y[j], eyy = eta_yy[j];
  const double* c = coef + ((long long)j * (D + 2) + a) * NW;
  double f[NW];
  for (int q = 0; q < NW; ++q) f[q] = c[q];
  for (int fi = 0; fi < D + 3; ++fi) f[o1 + 1 * (D + 3) + fi] = c[o1 + 1 * (D + 3) + fi] * ey;
  for (int g = 0; g < D + 1; ++g) {
    f[o2 + 1 * (D + 1) + g] = c[o2 + 1 * (D + 1) + g] * ey * ey;
    const int fi = g < D ? 1 + g : D + 2;
    f[o1 + 1 * (D + 3) + fi] += c[o2 + 1 * (D + 1) + g] * eyy;
  }
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k)
      if (i != k && (i == 1 || k == 1)) f[om + i * D + k] = c[om + i * D + k] * ey;
  double* o = out + ((long long)j * (D + 2) + a) * NW;
  for (int q = 0; q < NW; ++q) o[q] = f[q];
}

__global__ void k_split_pairs(const double* in, ffn* out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = ff_split(in[i]);
}

__global__ void k_to_float_tab(const double* in, float* out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// T's scaled difference split the same way: FP64 first order + FP32 rest
__device__ __forceinline__ void temperature_fast_body(const PointParams& P, double2* Tw, unsigned bidx, unsigned nb) {
  const int D = P.nz > 1 ? 3 : 2;
  const double e = *P.eps;
  const float ef = (float)e;
  const pw::ClosureK C = P.phys.C;
  for (long long pt = (long long)bidx * blockDim.x + threadIdx.x; pt < P.npts; pt += (long long)nb * blockDim.x) {
    const int j = row_of(P, pt);
    const double ip0 = P.btab[pw::bt_extra(D, pw::X_IP) * P.nbase + j];
    const double T0 = P.btab[pw::bt_val(D, D + 2) * P.nbase + j];
    const double2 wp = P.v[pt], ws = P.v[(long long)(D + 1) * P.npts + pt];
    double t[2];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
      const double q = (part ? wp.y : wp.x) * ip0, s = part ? ws.y : ws.x;
      const double X1 = fma(C.omig, q, s * C.icp);
      double r = T0 * X1;
      if (e != 0.0) {
        const float qf = (float)q;
        const float X2 = (float)C.omig * qf * pw::log1p_m1_over_f(ef * qf);
        const float X = (float)X1 + X2;
        r += (double)((float)T0 * fmaf(X, pw::expm1_m1_over_f(ef * X), X2));
      }
      t[part] = r;
    }
    Tw[pt] = make_double2(t[0], t[1]);
  }
}

__global__ void k_temperature_fast(const PointParams P, double2* Tw) {
  if (P.gate && *P.gate) return;
  temperature_fast_body(P, Tw, blockIdx.x, gridDim.x);
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
  double pref, igam, icp, R, gam, S;
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
    const double T = p / (rho * P.R);
    out(bt_val(D, D + 2), T);
    out(bt_val(D, D + 3), rho);
    const double c = sqrt(P.gam * p / rho);
    out(bt_extra(D, pw::X_IRHO), 1.0 / rho);
    out(bt_extra(D, pw::X_IP), 1.0 / p);
    out(bt_extra(D, pw::X_IT), 1.0 / T);
    out(bt_extra(D, pw::X_SQT), sqrt(T));
    out(bt_extra(D, pw::X_ITS), 1.0 / (T + P.S));
    out(bt_extra(D, pw::X_C), c);
    out(bt_extra(D, pw::X_RC), rho * c);
    out(bt_extra(D, pw::X_IRC), 1.0 / (rho * c));
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

static PackParams pack_params(StabHandle* h, double* btab) {
  const int D = h->dim;
  PackParams K{};
  K.q0 = h->d_q0;
  K.scratch = h->d_scratch;
  K.btab = btab;
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
  K.gam = h->gamma;
  K.S = h->S;
  return K;
}

// ---------------------------------------------------------------------------
// Batched J v: one launch per phase runs the work items (instance, block) of
// several problems of uneven size.  Item i owns the flat blocks
// [start[i], start[i+1]); a CTA finds its item by binary search, copies the
// item's parameters to shared memory and runs the single-problem body with
// its local block index, so every instance computes exactly what its own
// launch would.
// ---------------------------------------------------------------------------
struct NormItem {
  const double2* v;
  long long n;
  double* partial;
  unsigned* counter;
  double* out;
  double q0norm, fixed_eps;
  const int* gate;  // per-instance gate of a batched solver (nullable)
  int mode, pad;
};
struct TempItem {
  PointParams P;
  double2* Tw;
};
struct PointItem {
  PointParams P;
  const ffn* coefp;
  const float* btab_f;
};
static_assert(sizeof(PassParams) % 8 == 0 && sizeof(TempItem) % 8 == 0 && sizeof(PointItem) % 8 == 0,
              "items are copied to shared memory in 8-byte words");

// largest i with start[i] <= b (start[0] = 0, increasing)
__device__ __forceinline__ int batch_item(const int* __restrict__ start, int count, unsigned b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void copy_to_shared(void* dst, const void* src, size_t bytes) {
  const unsigned long long* s8 = (const unsigned long long*)src;
  unsigned long long* d8 = (unsigned long long*)dst;
  for (size_t k = threadIdx.x; k < bytes / 8; k += blockDim.x) d8[k] = __ldg(s8 + k);
}

__global__ void k_norm2_batch(const NormItem* __restrict__ items, const int* __restrict__ start, int count) {
  const int i = batch_item(start, count, blockIdx.x);
  const NormItem it = items[i];
  if (it.gate && *it.gate) return;
  const unsigned nb = (unsigned)(__ldg(start + i + 1) - __ldg(start + i));
  norm2_body(it.v, it.n, it.partial, it.counter, it.out, it.mode, it.q0norm, it.fixed_eps,
             blockIdx.x - (unsigned)__ldg(start + i), nb);
}

__global__ void k_temperature_fast_batch(const TempItem* __restrict__ items, const int* __restrict__ start, int count) {
  __shared__ TempItem sI;
  const int i = batch_item(start, count, blockIdx.x);
  copy_to_shared(&sI, items + i, sizeof(TempItem));
  __syncthreads();
  if (sI.P.gate && *sI.P.gate) return;
  const unsigned s0 = (unsigned)__ldg(start + i);
  temperature_fast_body(sI.P, sI.Tw, blockIdx.x - s0, (unsigned)__ldg(start + i + 1) - s0);
}

template <int D>
__global__ void __launch_bounds__(128, D == 2 ? 4 : 3)
    k_point_fast_batch(const PointItem* __restrict__ items, const int* __restrict__ start, int count) {
  __shared__ PointItem sI;
  const int i = batch_item(start, count, blockIdx.x);
  copy_to_shared(&sI, items + i, sizeof(PointItem));
  __syncthreads();
  if (sI.P.gate && *sI.P.gate) return;
  const unsigned s0 = (unsigned)__ldg(start + i);
  point_fast_body<D>(sI.P, sI.coefp, sI.btab_f, blockIdx.x - s0, (unsigned)__ldg(start + i + 1) - s0);
}

// line passes: item = (instance, axis, chunk of at most STAB_MAX_JOBS jobs);
// its blocks are (line block, job) with the line block fastest
template <bool FF>
__global__ void k_line_pass_batch(const PassParams* __restrict__ items, const int* __restrict__ start, int count) {
  __shared__ PassParams sP;
  const int i = batch_item(start, count, blockIdx.x);
  copy_to_shared(&sP, items + i, sizeof(PassParams));
  __syncthreads();
  const unsigned local = blockIdx.x - (unsigned)__ldg(start + i);
  const unsigned nbx = (unsigned)((sP.nlines + sP.L - 1) / sP.L);
  line_pass_body<FF>(sP, local % nbx, local / nbx);
}

template <bool FF>
__global__ void __launch_bounds__(kCompactMaxThreads)
    k_line_pass_compact_batch(const PassParams* __restrict__ items, const int* __restrict__ start, int count) {
  __shared__ PassParams sP;
  const int i = batch_item(start, count, blockIdx.x);
  copy_to_shared(&sP, items + i, sizeof(PassParams));
  __syncthreads();
  const unsigned local = blockIdx.x - (unsigned)__ldg(start + i);
  const unsigned nbx = (unsigned)((sP.nlines + sP.L - 1) / sP.L);
  line_pass_compact_body<FF>(sP, local % nbx, local / nbx);
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
pw::Phys phys_of(const StabHandle* h) {
  pw::Phys p;
  p.gamma = h->gamma;
  p.R = h->R;
  p.cp = h->cp;
  p.Pr = h->Pr;
  p.S = h->S;
  p.Re = h->Re;
  p.bulk = h->bulk;
  p.C.ig = 1.0 / h->gamma;
  p.C.omig = 1.0 - 1.0 / h->gamma;
  p.C.icp = 1.0 / h->cp;
  p.visc = h->visc;
  return p;
}

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
    // FP32 part of the warm-up: its relative error 2^-24 is damped by |r|^Wn <= 2^-32
    A.Wn[kind] = (int)std::ceil(32.0 * std::log(2.0) / -std::log(std::fabs(r))) + 1;
    if (A.periodic) {
      const double c = -al / r;  // circulant = c (1 - r S^-1)(1 - r S)
      for (int t = 0; t < n; ++t) { l[t] = -r; dinv[t] = 1.0 / c; m[t] = -r; }
      A.pdinv[kind] = 1.0 / c;
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
        const double lt = a[t] / d, dprev = d;
        d = b[t] - lt * cc[t - 1];
        dinv[t] = 1.0 / d;
        m[t] = cc[t] / d;
        l[t] = lt * dprev * dinv[t];  // recurrence of the scaled forward sweep g'_t = g_t / d_t
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

// Parameters and launch shape of one axis's line pass for njobs jobs (the job
// list itself is filled by the caller, STAB_MAX_JOBS per launch).
static cudaError_t pass_shape(StabHandle* h, int axis, const PassParams& base_params, size_t njobs,
                              long long contiguous_lines, PassParams& P, int& threads, size_t& smem) {
  P = base_params;
  const AxisTables& A = h->ax[axis];
  P.axis = axis;
  P.n = A.n;
  P.nx = h->nx;
  P.ny = h->ny;
  P.periodic = A.periodic;
  P.h = A.h;
  P.tab[0] = A.tab[0];
  P.tab[1] = A.tab[1];
  P.tabf[0] = A.tabf[0];
  P.tabf[1] = A.tabf[1];
  P.Wn[0] = A.Wn[0];
  P.Wn[1] = A.Wn[1];

  P.K[0] = A.K[0];
  P.K[1] = A.K[1];

  P.stride = axis == 0 ? 1 : axis == 1 ? h->nx : (long long)h->nx * h->ny;
  P.nlines = h->npts / A.n;
  if (contiguous_lines >= 0) {  // lines stored back to back (line l at l * n), this axis's scheme
    P.axis = 0;
    P.nx = A.n;
    P.stride = 1;
    P.nlines = contiguous_lines;
  }
  // interior weights: first (a/2h, b/4h), second (a/h^2, b/4h^2)
  P.c1[0] = (14.0 / 9.0) / (2.0 * A.h);
  P.c2[0] = (1.0 / 9.0) / (4.0 * A.h);
  P.c1[1] = (12.0 / 11.0) / (A.h * A.h);
  P.c2[1] = (3.0 / 11.0) / (4.0 * A.h * A.h);
  if (A.periodic)  // the constant row scale 1/c of the factorised circulant
    for (int k = 0; k < 2; ++k) {
      P.c1[k] *= A.pdinv[k];
      P.c2[k] *= A.pdinv[k];
    }
  for (int k = 0; k < 2; ++k) {  // pair split of the weights (host rounding to nearest)
    P.c1h[k] = (float)P.c1[k];
    P.c1l[k] = (float)(P.c1[k] - (double)P.c1h[k]);
    P.c2h[k] = (float)P.c2[k];
    P.c2l[k] = (float)(P.c2[k] - (double)P.c2h[k]);
  }

  const int n = A.n;
  if (n > 2048) return cudaErrorInvalidValue;
  // launch shape: C points per sweep chunk, L lines per CTA, KP kinds at
  // once.  Either tuned (stab_autotune) or by default: on small grids
  // (latency matters) both kinds side by side in chunks of 16, at most two
  // lines per CTA and fewer so that the CTAs cover the SMs (but at least a
  // warp of threads); on larger grids the compact layout in chunks of 32 with
  // up to four lines per CTA (shared memory bounds occupancy there).
  const LineCfg cfg = contiguous_lines >= 0 ? LineCfg{} : h->line_cfg[axis];
  const long long fill = (P.nlines * (long long)njobs + 2 * 152 - 1) / (2 * 152);
  const bool small = fill <= 4;
  P.C = cfg.C > 0 ? cfg.C : (small || n < 64 ? 16 : 32);
  P.nchunks = (n + P.C - 1) / P.C;
  P.LS = n + (n >> 5) + 1;
  const long long LS = P.LS;
  P.KP = cfg.kp > 0 ? cfg.kp : (small ? 2 : 3);
  const int tpl = (P.KP == 2 ? 4 : 2) * P.nchunks;  // threads per line
  const int max_threads = P.KP == 3 ? kCompactMaxThreads : 1024;
  if (tpl > max_threads) return cudaErrorInvalidValue;
  const long long smem_line = (P.KP == 3 ? 2 : 2 + 2 * P.KP) * 8 * LS;
  const int maxL = std::min<long long>(std::min(max_threads / tpl, 32), (kLineSmemMax - kLineSmemExtra) / smem_line);
  if (maxL < 1) return cudaErrorInvalidValue;
  int L;
  if (cfg.L > 0) {
    L = std::min(cfg.L, maxL);
  } else {
    // compact layout: at least four lines and a CTA of about 128 threads (short lines)
    const int Lc = std::max(4, (128 + tpl - 1) / tpl);
    L = std::min<long long>(std::min<long long>(maxL, 98304 / smem_line), P.KP == 3 ? Lc : 2);
    const int Lwarp = (32 + tpl - 1) / tpl;
    if (L > fill) L = (int)std::min<long long>(maxL, std::max<long long>(fill, Lwarp));
  }
  if (L < 1) L = 1;
  P.L = L;
  P.divn = make_fastdiv((unsigned)n);
  P.divL = make_fastdiv((unsigned)L);
  P.divnx = make_fastdiv((unsigned)P.nx);
  threads = tpl * L;
  threads = ((threads + 31) / 32) * 32;
  smem = (size_t)smem_line * L + kLineSmemExtra;
  return cudaSuccess;
}

static cudaError_t run_pass(StabHandle* h, int axis, const PassParams& base_params, const std::vector<LineJob>& jobs,
                            long long contiguous_lines = -1) {
  if (jobs.empty()) return cudaSuccess;
  PassParams P;
  int threads = 0;
  size_t smem = 0;
  const cudaError_t e = pass_shape(h, axis, base_params, jobs.size(), contiguous_lines, P, threads, smem);
  if (e != cudaSuccess) return e;
  const int L = P.L;
  for (size_t j0 = 0; j0 < jobs.size(); j0 += STAB_MAX_JOBS) {
    P.njobs = (int)std::min<size_t>(STAB_MAX_JOBS, jobs.size() - j0);
    for (int q = 0; q < P.njobs; ++q) P.job[q] = jobs[j0 + q];
    dim3 grid((unsigned)((P.nlines + L - 1) / L), (unsigned)P.njobs);
    if (P.KP == 3) {
      if (P.ff) k_line_pass_compact<true><<<grid, threads, smem, h->stream>>>(P);
      else k_line_pass_compact<false><<<grid, threads, smem, h->stream>>>(P);
    } else {
      if (P.ff) k_line_pass<true><<<grid, threads, smem, h->stream>>>(P);
      else k_line_pass<false><<<grid, threads, smem, h->stream>>>(P);
    }
  }
  return cudaGetLastError();
}

// jobs of the line pass along axis ax for field sources src[f] (f = 0..D+2):
// first (and second) derivatives of every field, plus the mixed derivatives
// formed from y derivatives (z pass: d/dz of d/dy v, w; x pass: d/dx of d/dy
// u, v and, in 3-D, of d/dz u, w)
static void axis_jobs(StabHandle* h, int ax, const double2* const* src, std::vector<LineJob>& jobs) {
  const int D = h->dim;
  const Slots& S = h->slots;
  double2* sc = h->d_scratch;
  auto slot = [&](int s) -> double2* { return s >= 0 ? sc + (long long)s * h->npts : nullptr; };
  const int nf = h->visc ? D + 3 : D + 2;
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
  if (!h->visc) return;
  if (ax == 2) {
    jobs.push_back(LineJob{slot(S.d1[1][2]), slot(S.mix[2][1]), nullptr});
    jobs.push_back(LineJob{slot(S.d1[1][3]), slot(S.mix[1][2]), nullptr});
  } else if (ax == 0) {
    jobs.push_back(LineJob{slot(S.d1[1][2]), slot(S.mix[0][1]), nullptr});
    jobs.push_back(LineJob{slot(S.d1[1][1]), slot(S.mix[1][0]), nullptr});
    if (D == 3) {
      jobs.push_back(LineJob{slot(S.d1[2][3]), slot(S.mix[0][2]), nullptr});
      jobs.push_back(LineJob{slot(S.d1[2][1]), slot(S.mix[2][0]), nullptr});
    }
  }
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// The reduced operator's base table: the base fields' derivatives taken with
// second-order explicit differences (Sec. "Numerical experiments", the
// non-compact lower-order discretisation proposed for the preconditioner):
// f'_i = (f_{i+1} - f_{i-1})/(2h), f''_i = (f_{i+1} - 2 f_i + f_{i-1})/h^2,
// on a bounded line the end rows second-order one-sided,
// f'_0 = (-3 f_0 + 4 f_1 - f_2)/(2h), f''_0 = (2 f_0 - 5 f_1 + 4 f_2 - f_3)/h^2
// (mirrored at the far end, the first with a sign change).  Derivatives in the
// computational coordinate, into the same slots as the compact passes.
// ---------------------------------------------------------------------------
__global__ void k_low_deriv(const double2* in, double2* out1, double2* out2, int axis, int n, double hh, int periodic,
                            int nx, int ny, long long npts) {
  const long long st = axis == 0 ? 1 : axis == 1 ? nx : (long long)nx * ny;
  for (long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x; pt < npts; pt += (long long)gridDim.x * blockDim.x) {
    const int i = axis == 0 ? (int)(pt % nx) : axis == 1 ? (int)((pt / nx) % ny) : (int)(pt / ((long long)nx * ny));
    auto f = [&](int k) {
      if (periodic) k = (k % n + n) % n;
      return in[pt + (long long)(k - i) * st];
    };
    double2 d1, d2;
    if (periodic || (i > 0 && i < n - 1)) {
      const double2 fp = f(i + 1), fm = f(i - 1), f0 = f(i);
      d1 = make_double2((fp.x - fm.x) / (2.0 * hh), (fp.y - fm.y) / (2.0 * hh));
      d2 = make_double2((fp.x - 2.0 * f0.x + fm.x) / (hh * hh), (fp.y - 2.0 * f0.y + fm.y) / (hh * hh));
    } else {
      const int sg = i == 0 ? 1 : -1;  // direction into the line
      const double2 a0 = f(i), a1 = f(i + sg), a2 = f(i + 2 * sg), a3 = f(i + 3 * sg);
      const double s1 = sg / (2.0 * hh);
      d1 = make_double2((-3.0 * a0.x + 4.0 * a1.x - a2.x) * s1, (-3.0 * a0.y + 4.0 * a1.y - a2.y) * s1);
      d2 = make_double2((2.0 * a0.x - 5.0 * a1.x + 4.0 * a2.x - a3.x) / (hh * hh),
                        (2.0 * a0.y - 5.0 * a1.y + 4.0 * a2.y - a3.y) / (hh * hh));
    }
    if (out1) out1[pt] = d1;
    if (out2) out2[pt] = d2;
  }
}

cudaError_t jv_reduced_base_table(StabHandle* h, double* btab) {
  const int D = h->dim;
  cudaError_t err;
  double2* bv;
  if ((err = dalloc(h, &bv, (size_t)(h->nv + 1) * h->npts * sizeof(double2))) != cudaSuccess) return err;
  double2* bT = bv + (long long)h->nv * h->npts;
  const int thr = 256;
  k_base_fields<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(h->d_q0, h->npts, h->nv, h->R, 1.0 / h->gamma,
                                                                1.0 / h->cp, h->R, bv, bT);
  const double2* src[6];
  for (int f = 0; f < D + 2; ++f) src[f] = bv + (long long)f * h->npts;
  src[D + 2] = bT;
  static const int order[3] = {1, 2, 0};  // y and z first: the mixed derivatives take their outputs
  for (int q = 0; q < 3 && (err = cudaGetLastError()) == cudaSuccess; ++q) {
    const int ax = order[q];
    if (ax >= D) continue;
    std::vector<LineJob> jobs;
    axis_jobs(h, ax, src, jobs);
    for (const LineJob& J : jobs)
      k_low_deriv<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(J.in, J.out1, J.out2, ax, h->ax[ax].n, h->ax[ax].h,
                                                                 h->ax[ax].periodic, h->nx, h->ny, h->npts);
  }
  if (err == cudaSuccess) {
    PackParams K = pack_params(h, btab);
    k_pack_base<<<grid_for(h->nbase, thr), thr, 0, h->stream>>>(K);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
  dfree(h, bv);
  return err;
}

// all derivative passes for field sources src[f] (f = 0..D+2): y, then z,
// then x (the mixed derivatives need the y and z passes)
static cudaError_t run_derivatives(StabHandle* h, const double2* const* src, int ff) {
  PassParams P{};
  P.gate = h->gate;
  P.ff = ff;
  static const int order[3] = {1, 2, 0};
  static const int phase[3] = {STAB_PHASE_LINE_Y, STAB_PHASE_LINE_Z, STAB_PHASE_LINE_X};
  for (int q = 0; q < 3; ++q) {
    const int ax = order[q];
    if (ax >= h->dim) continue;
    std::vector<LineJob> jobs;
    axis_jobs(h, ax, src, jobs);
    const int ts = phase_begin(h, phase[q]);
    cudaError_t err = run_pass(h, ax, P, jobs);
    if (err != cudaSuccess) return err;
    phase_end(h, ts);
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Autotuner of the line-pass launch shape (C, L) per axis: every admissible
// candidate is timed with CUDA events on this handle's jobs, the fastest is
// kept in the handle and in a process-wide cache keyed by device, line length,
// line count, job count and boundary type.  C changes where the sweeps'
// warm-up starts, so results may differ at the rounding level between shapes;
// L does not change any result.
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
  int dev, n, njobs, periodic, ff;
  long long nlines;
  bool operator<(const TuneKey& o) const {
    if (dev != o.dev) return dev < o.dev;
    if (ff != o.ff) return ff < o.ff;
    if (n != o.n) return n < o.n;
    if (nlines != o.nlines) return nlines < o.nlines;
    if (njobs != o.njobs) return njobs < o.njobs;
    return periodic < o.periodic;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, LineCfg> g_tune;
}  // namespace

static TuneKey tune_key(StabHandle* h, int ax, int njobs) {
  TuneKey k;
  cudaGetDevice(&k.dev);
  k.n = h->ax[ax].n;
  k.nlines = h->npts / h->ax[ax].n;
  k.njobs = njobs;
  k.periodic = h->ax[ax].periodic;
  k.ff = h->stencil_ff;
  return k;
}

cudaError_t jv_autotune(StabHandle* h, int force, double* ms_out) {
  const int D = h->dim;
  double2* tmp = nullptr;
  cudaError_t err = cudaSuccess;
  for (int ax = 0; ax < D && err == cudaSuccess; ++ax) {
    std::vector<LineJob> jobs;
    const double2* src[6];
    if (!tmp) {
      if ((err = dalloc(h, &tmp, (size_t)h->n * sizeof(double2))) != cudaSuccess) break;
      if ((err = cudaMemsetAsync(tmp, 0, (size_t)h->n * sizeof(double2), h->stream)) != cudaSuccess) break;
    }
    for (int f = 0; f < D + 2; ++f) src[f] = tmp + (long long)f * h->npts;
    src[D + 2] = h->d_scratch + (long long)h->slots.Tw * h->npts;
    axis_jobs(h, ax, src, jobs);
    const TuneKey key = tune_key(h, ax, (int)jobs.size());
    if (!force) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        h->line_cfg[ax] = it->second;
        if (ms_out) ms_out[ax] = -1.0;
        continue;
      }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    PassParams P{};
    P.ff = h->stencil_ff;
    LineCfg best{};
    double best_ms = 1e300;
    const int n = h->ax[ax].n;
    for (int kp : {1, 2, 3}) {
      for (int C : {16, 32, 64}) {
        if (C > 16 && C >= 2 * n) continue;
        for (int L : {1, 2, 4, 8, 16, 32}) {
          const int nch = (n + C - 1) / C;
          const long long LS = n + (n >> 5) + 1;
          const int tpl = (kp == 2 ? 4 : 2) * nch;
          const int planes = kp == 3 ? 2 : 2 + 2 * kp;
          if (tpl * L > (kp == 3 ? kCompactMaxThreads : 1024) || planes * 8 * LS * L + kLineSmemExtra > kLineSmemMax)
            continue;
          h->line_cfg[ax] = LineCfg{C, L, kp};
          if (run_pass(h, ax, P, jobs) != cudaSuccess) {  // a shape this device cannot launch: skip it
            cudaGetLastError();
            continue;
          }
          // three back-to-back launches per sample (less launch and clock noise), best of five samples
          float best_t = 1e30f;
          for (int r = 0; r < 5 && err == cudaSuccess; ++r) {
            cudaEventRecord(e0, h->stream);
            for (int q = 0; q < 3 && err == cudaSuccess; ++q) err = run_pass(h, ax, P, jobs);
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best_t = std::min(best_t, t / 3.0f);
          }
          if (err != cudaSuccess) break;
          if (best_t < best_ms) { best_ms = best_t; best = LineCfg{C, L, kp}; }
        }
        if (err != cudaSuccess) break;
      }
      if (err != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) break;
    h->line_cfg[ax] = best;
    if (ms_out) ms_out[ax] = best_ms;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  if (tmp) {
    cudaStreamSynchronize(h->stream);
    dfree(h, tmp);
  }
  if (err != cudaSuccess) for (int ax = 0; ax < 3; ++ax) h->line_cfg[ax] = LineCfg{};
  return err;
}

// cache file: one line per entry, "n nlines njobs periodic C L kinds ff" (ff: pair
// stencil; a line without it is an FP64-stencil entry); entries are applied to the
// current device when loaded
int jv_tune_save(const char* path) {
  FILE* f = std::fopen(path, "w");
  if (!f) return -1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& kv : g_tune)
    std::fprintf(f, "%d %lld %d %d %d %d %d %d\n", kv.first.n, kv.first.nlines, kv.first.njobs, kv.first.periodic,
                 kv.second.C, kv.second.L, kv.second.kp, kv.first.ff);
  std::fclose(f);
  return (int)g_tune.size();
}

int jv_tune_load(const char* path) {
  FILE* f = std::fopen(path, "r");
  if (!f) return -1;
  int dev = 0;
  cudaGetDevice(&dev);
  int count = 0;
  TuneKey k;
  LineCfg c;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    k.ff = 0;
    const int got = std::sscanf(line, "%d %lld %d %d %d %d %d %d", &k.n, &k.nlines, &k.njobs, &k.periodic, &c.C, &c.L,
                                &c.kp, &k.ff);
    if (got < 7) continue;
    if (c.C < 1 || c.L < 1 || c.kp < 1 || c.kp > 3 || k.n < 1 || (k.ff != 0 && k.ff != 1))
      continue;
    k.dev = dev;
    g_tune[k] = c;
    ++count;
  }
  std::fclose(f);
  return count;
}

// apply cached shapes (if any) to a new handle
void jv_tune_apply_cached(StabHandle* h) {
  const double2* src[6] = {};
  for (int ax = 0; ax < h->dim; ++ax) {
    std::vector<LineJob> jobs;
    axis_jobs(h, ax, src, jobs);
    const TuneKey key = tune_key(h, ax, (int)jobs.size());
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) h->line_cfg[ax] = it->second;
  }
}

static PointParams point_params(StabHandle* h, const double2* v) {
  PointParams P{};
  P.gate = h->gate;
  P.divnx = make_fastdiv((unsigned)h->nx);
  P.divny = make_fastdiv((unsigned)h->ny);
  P.v = v;
  P.scratch = h->d_scratch;
  P.npts = h->npts;
  P.nx = h->nx;
  P.ny = h->ny;
  P.nz = h->nz;
  P.homog = h->homog;
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
  P.eta_y_f = P.eta_y;
  P.eta_yy_f = P.eta_yy;
  P.bcflags = h->d_bcflags;
  P.eps = h->d_eps;
  P.phys = phys_of(h);
  return P;
}

cudaError_t launch_norm2(StabHandle* h, const double2* v, long long n, double* d_out, int mode) {
  // block count depends on n only, so the summation order is reproducible
  long long nb = (n + 1023) / 1024;
  if (nb > h->red_blocks) nb = h->red_blocks;
  if (nb < 1) nb = 1;
  k_norm2<<<(int)nb, 256, 0, h->stream>>>(v, n, h->d_red, (unsigned*)(h->d_red + h->red_blocks + 8), d_out, mode,
                                         h->q0norm, h->opts.eps, h->gate);
  return cudaGetLastError();
}

cudaError_t jv_setup(StabHandle* h, const double* q0_host) {
  const int D = h->dim;
  cudaError_t err;
  // set once per handle (current device), never during a stream capture
  const void* line_kernels[4] = {(const void*)k_line_pass<false>, (const void*)k_line_pass<true>,
                                 (const void*)k_line_pass_compact<false>, (const void*)k_line_pass_compact<true>};
  for (const void* k : line_kernels)
    if ((err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLineSmemMax)) != cudaSuccess)
      return err;
  make_slots(h);
  // axis tables: x (0) periodic, y (1) bounded in eta, z (2) periodic
  const int lens[3] = {h->nx, h->ny, h->nz};
  for (int ax = 0; ax < 3; ++ax) {
    AxisTables& A = h->ax[ax];
    A.n = lens[ax];
    A.periodic = ax != 1;
    A.h = ax == 0 ? h->lx / h->nx : ax == 1 ? 1.0 / (h->ny - 1) : (D == 3 ? h->lz / h->nz : 1.0);
    A.tab[0] = A.tab[1] = nullptr;
    A.tabf[0] = A.tabf[1] = nullptr;
    if (ax >= D) continue;
    std::vector<double> host;
    fill_axis_tables(A, host);
    double* d;
    if ((err = dalloc(h, &d, host.size() * sizeof(double))) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(d, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) return err;
    A.tab[0] = d;
    A.tab[1] = d + 3 * A.n;
    std::vector<float> hf((size_t)4 * A.n);
    for (int k = 0; k < 2; ++k)
      for (int t = 0; t < A.n; ++t) {
        hf[(size_t)k * 2 * A.n + t] = (float)host[(size_t)k * 3 * A.n + t];               // l'
        hf[(size_t)k * 2 * A.n + A.n + t] = (float)host[(size_t)k * 3 * A.n + 2 * A.n + t];  // m
      }
    float* df;
    if ((err = dalloc(h, &df, hf.size() * sizeof(float))) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(df, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
      return err;
    if ((err = cudaStreamSynchronize(h->stream)) != cudaSuccess) return err;  // host vectors go out of scope
    A.tabf[0] = df;
    A.tabf[1] = df + 2 * A.n;
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
    if ((err = dalloc(h, &h->d_metric, met.size() * sizeof(double))) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(h->d_metric, met.data(), met.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) return err;
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
    if ((err = dalloc(h, &h->d_bcflags, fl.size())) != cudaSuccess) return err;
    if ((err = cudaMemcpyAsync(h->d_bcflags, fl.data(), fl.size(), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess) return err;
  }
  // scratch, reductions, eps
  if ((err = dalloc(h, &h->d_scratch, (size_t)h->slots.count * h->npts * sizeof(double2))) != cudaSuccess) return err;
  h->red_blocks = 1024;
  if ((err = dalloc(h, &h->d_red, (h->red_blocks + 64) * sizeof(double))) != cudaSuccess) return err;
  h->d_eps = h->d_red + h->red_blocks;
  // completion counter of the one-launch norm (k_norm2) at d_red + red_blocks + 8: starts at zero
  if ((err = cudaMemsetAsync(h->d_red + h->red_blocks, 0, 64 * sizeof(double), h->stream)) != cudaSuccess) return err;
  k_set_scalar<<<1, 1, 0, h->stream>>>(h->d_eps, 0.0);
  // base tables: derivatives of the base fields through the same passes
  const int nbt = bt_count(D);
  if ((err = dalloc(h, &h->d_btab, (size_t)nbt * h->nbase * sizeof(double))) != cudaSuccess) return err;
  double2* bv;
  if ((err = dalloc(h, &bv, (size_t)(h->nv + 1) * h->npts * sizeof(double2))) != cudaSuccess) return err;
  double2* bT = bv + (long long)h->nv * h->npts;
  int thr = 256;
  k_base_fields<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(h->d_q0, h->npts, h->nv, h->R, 1.0 / h->gamma,
                                                                1.0 / h->cp, h->R, bv, bT);
  const double2* src[6];
  for (int f = 0; f < D + 2; ++f) src[f] = bv + (long long)f * h->npts;
  src[D + 2] = bT;
  if ((err = run_derivatives(h, src, 0)) != cudaSuccess) return err;  // base tables: FP64 right-hand sides
  PackParams K = pack_params(h, h->d_btab);
  k_pack_base<<<grid_for(h->nbase, thr), thr, 0, h->stream>>>(K);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (h->homog) {
    const int nw = pw::nw_inputs(D);
    if ((err = dalloc(h, &h->d_coef, (size_t)h->ny * (D + 2) * nw * sizeof(double))) != cudaSuccess) return err;
    PointParams PP = point_params(h, nullptr);
    if (D == 2) k_coeffs<2><<<h->ny, 32, 0, h->stream>>>(PP, h->d_coef);
    else k_coeffs<3><<<h->ny, 64, 0, h->stream>>>(PP, h->d_coef);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if ((err = dalloc(h, &h->d_coef_f, (size_t)h->ny * (D + 2) * nw * sizeof(double))) != cudaSuccess) return err;
    if (D == 2) k_coeffs_fold<2><<<h->ny, 32, 0, h->stream>>>(h->d_coef, h->d_metric, h->d_metric + h->ny, h->ny, h->d_coef_f);
    else k_coeffs_fold<3><<<h->ny, 32, 0, h->stream>>>(h->d_coef, h->d_metric, h->d_metric + h->ny, h->ny, h->d_coef_f);
    const long long ncf = (long long)h->ny * (D + 2) * nw;
    if ((err = dalloc(h, &h->d_coef_p, ncf * sizeof(ffn))) != cudaSuccess) return err;
    k_split_pairs<<<64, 256, 0, h->stream>>>(h->d_coef_f, h->d_coef_p, ncf);
    const long long nbt = (long long)bt_count(D) * h->nbase;
    if ((err = dalloc(h, &h->d_btab_f, nbt * sizeof(float))) != cudaSuccess) return err;
    k_to_float_tab<<<64, 256, 0, h->stream>>>(h->d_btab, h->d_btab_f, nbt);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  if ((err = cudaStreamSynchronize(h->stream)) != cudaSuccess) return err;
  dfree(h, bv);
  return cudaSuccess;
}

// Dense 1-D derivative matrices of an axis, column-major: out1[l * n + t] =
// (D e_l)_t and out2 likewise for the second derivative, computed by the
// same line sweeps as the operator.
cudaError_t jv_derivative_matrices(StabHandle* h, int axis, double2* work, double2* out1, double2* out2) {
  const int n = h->ax[axis].n;
  std::vector<double2> eye((size_t)n * n, make_double2(0.0, 0.0));
  for (int l = 0; l < n; ++l) eye[(size_t)l * n + l] = make_double2(1.0, 0.0);
  cudaError_t e = cudaMemcpyAsync(work, eye.data(), eye.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return e;
  std::vector<LineJob> jobs{LineJob{work, out1, out2}};
  PassParams P{};
  if ((e = run_pass(h, axis, P, jobs, n)) != cudaSuccess) return e;
  return cudaStreamSynchronize(h->stream);  // eye must outlive the copy
}

cudaError_t jv_apply(StabHandle* h, const double2* v, double2* out, double2 shift, int eps_mode) {
  cudaError_t err;
  if (eps_mode == 2) {
    if (h->last_eps_mode != 2) k_set_scalar<<<1, 1, 0, h->stream>>>(h->d_eps, 0.0);
  } else {
    const int ts = phase_begin(h, STAB_PHASE_EPS);
    if ((err = launch_norm2(h, v, h->n, h->d_eps, 2)) != cudaSuccess) return err;
    phase_end(h, ts);
  }
  h->last_eps_mode = eps_mode;
  PointParams P = point_params(h, v);
  P.out = out;
  P.shift = shift;
  double2* Tw = h->d_scratch + (long long)h->slots.Tw * h->npts;
  const int thr = 128;
  const bool fast = h->homog && h->d_coef && !h->force_dn_path;
  if (h->visc) {
    const int ts = phase_begin(h, STAB_PHASE_TEMPERATURE);
    if (fast) k_temperature_fast<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P, Tw);
    else k_temperature<<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P, Tw);
    phase_end(h, ts);
  }
  const int D = h->dim;
  const double2* src[6];
  for (int f = 0; f < D + 2; ++f) src[f] = v + (long long)f * h->npts;
  src[D + 2] = Tw;
  if ((err = run_derivatives(h, src, h->stencil_ff)) != cudaSuccess) return err;
  const int tp = phase_begin(h, STAB_PHASE_POINTWISE);
  if (fast) {
    if (D == 2) k_point_fast<2><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P, h->d_coef_p, h->d_btab_f);
    else k_point_fast<3><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P, h->d_coef_p, h->d_btab_f);
  } else {
    if (D == 2) k_point<2><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P);
    else k_point<3><<<grid_for(h->npts, thr), thr, 0, h->stream>>>(P);
  }
  phase_end(h, tp);
  h->stats.jv_calls++;
  return cudaGetLastError();
}

// ||v||_2 on an explicit stream with caller-provided partials (nb blocks,
// fixed by the caller so the summation order is reproducible).
cudaError_t launch_norm2_stream(cudaStream_t st, const double2* v, long long n, double* partial, int nb, double* d_out) {
  k_norm2_partial<<<nb, 256, 0, st>>>(v, n, partial, nullptr);
  k_norm2_final<<<1, 32, 0, st>>>(partial, nb, d_out, 1, 0.0, 0.0, nullptr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched J v over several handles (uneven grids): the per-instance items of
// every phase are built on the host, copied to device memory in one transfer
// (from a pinned staging buffer guarded by an event), and each phase is one
// launch per kernel variant for all instances.
// ---------------------------------------------------------------------------
// Copy a parameter image to the batch's device buffer: through the pinned
// staging buffer, once the previous transfer out of it has completed.
cudaError_t batch_stage(stab_jv_batch_s* B, const BatchImage& im) {
  if (im.overflow) return cudaErrorInvalidValue;
  const size_t bytes = im.bytes.size();
  cudaError_t e;
  if ((e = cudaEventSynchronize(B->copied)) != cudaSuccess) return e;
  if (bytes > B->h_cap) {
    if (B->h_buf) cudaFreeHost(B->h_buf);
    B->h_buf = nullptr;
    B->h_cap = 0;
    if ((e = cudaHostAlloc(&B->h_buf, bytes, cudaHostAllocDefault)) != cudaSuccess) return e;
    B->h_cap = bytes;
  }
  if (bytes > B->d_cap) {
    if (B->d_buf) cudaFreeAsync(B->d_buf, B->stream);
    B->d_buf = nullptr;
    B->d_cap = 0;
    if ((e = dev_alloc_stream(B->device, B->stream, &B->d_buf, bytes)) != cudaSuccess) return e;
    B->d_cap = bytes;
  }
  std::memcpy(B->h_buf, im.bytes.data(), bytes);
  if ((e = cudaMemcpyAsync(B->d_buf, B->h_buf, bytes, cudaMemcpyHostToDevice, B->stream)) != cudaSuccess) return e;
  return cudaEventRecord(B->copied, B->stream);
}

// distinct handle streams other than the batch's own
static std::vector<cudaStream_t> batch_handle_streams(const stab_jv_batch_s* B) {
  std::vector<cudaStream_t> out;
  for (const StabHandle* h : B->hs)
    if (h->stream != B->stream && std::find(out.begin(), out.end(), h->stream) == out.end()) out.push_back(h->stream);
  return out;
}

cudaError_t batch_order_begin(stab_jv_batch_s* B) {
  for (cudaStream_t s : batch_handle_streams(B)) {
    cudaError_t e = cudaEventRecord(B->order, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->order, 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t batch_order_end(stab_jv_batch_s* B) {
  const std::vector<cudaStream_t> ss = batch_handle_streams(B);
  if (ss.empty()) return cudaSuccess;
  cudaError_t e = cudaEventRecord(B->order, B->stream);
  for (cudaStream_t s : ss)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, B->order, 0);
  return e;
}

static cudaError_t jv_batch_attributes() {
  const void* ks[4] = {(const void*)k_line_pass_batch<false>, (const void*)k_line_pass_batch<true>,
                       (const void*)k_line_pass_compact_batch<false>, (const void*)k_line_pass_compact_batch<true>};
  for (const void* k : ks) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLineSmemMax);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Parameter-image sections of one batched J v (every phase, one section per
// kernel variant) for the instances hs: v[i] -> out[i] = J_i v[i] - shift_i v[i].
// gates (nullable, or per instance nullable): the instance's work is skipped
// while *gates[i] != 0 (batched solvers drop converged instances this way).
cudaError_t jv_batch_plan(const std::vector<StabHandle*>& hs, const double2* const* v, double2* const* out,
                          const double2* shifts, const int* const* gates, BatchImage& im, JvBatchPlan& plan) {
  const int count = (int)hs.size();
  // 1. epsilon: one norm item per epsilon-quotient instance
  std::vector<NormItem> norms;
  std::vector<int> norm_blocks;
  // 2. temperature differences (viscous instances)
  std::vector<TempItem> temps;
  std::vector<int> temp_blocks;
  // 4. pointwise assembly, per dimension
  std::vector<PointItem> points[2];
  std::vector<int> point_blocks[2];
  plan.zero_eps.clear();
  for (int i = 0; i < count; ++i) {
    StabHandle* h = hs[i];
    const int* gate = gates ? gates[i] : nullptr;
    if (h->opts.eps_mode != 2) {
      long long nb = (h->n + 1023) / 1024;
      nb = std::max<long long>(1, std::min<long long>(nb, h->red_blocks));
      NormItem it{};
      it.v = v[i];
      it.n = h->n;
      it.partial = h->d_red;
      it.counter = (unsigned*)(h->d_red + h->red_blocks + 8);
      it.out = h->d_eps;
      it.q0norm = h->q0norm;
      it.fixed_eps = h->opts.eps;
      it.mode = 2;
      it.gate = gate;
      norms.push_back(it);
      norm_blocks.push_back((int)nb);
    } else {
      plan.zero_eps.push_back(h->d_eps);
    }
    PointParams P = point_params(h, v[i]);
    P.gate = gate;
    P.out = out[i];
    P.shift = shifts ? shifts[i] : make_double2(0.0, 0.0);
    double2* Tw = h->d_scratch + (long long)h->slots.Tw * h->npts;
    if (h->visc) {
      temps.push_back(TempItem{P, Tw});
      temp_blocks.push_back(grid_for(h->npts, 128));
    }
    points[h->dim - 2].push_back(PointItem{P, h->d_coef_p, h->d_btab_f});
    point_blocks[h->dim - 2].push_back(grid_for(h->npts, 128));
  }
  plan.norm = im.section(norms, norm_blocks, 256, 0);
  plan.temp = im.section(temps, temp_blocks, 128, 0);
  // 3. line passes y, z, x; per axis one section per kernel variant (main /
  // compact, FP64 / pair right-hand sides)
  static const int order[3] = {1, 2, 0};
  for (int q = 0; q < 3; ++q) {
    const int ax = order[q];
    std::vector<PassParams> items[4];
    std::vector<int> blocks[4];
    int threads[4] = {0, 0, 0, 0};
    size_t smem[4] = {0, 0, 0, 0};
    for (int i = 0; i < count; ++i) {
      StabHandle* h = hs[i];
      if (ax >= h->dim) continue;
      const int D = h->dim;
      const double2* src[6];
      for (int f = 0; f < D + 2; ++f) src[f] = v[i] + (long long)f * h->npts;
      src[D + 2] = h->d_scratch + (long long)h->slots.Tw * h->npts;
      std::vector<LineJob> jobs;
      axis_jobs(h, ax, src, jobs);
      if (jobs.empty()) continue;
      PassParams base{};
      base.ff = h->stencil_ff;
      base.gate = gates ? gates[i] : nullptr;
      PassParams P;
      int thr = 0;
      size_t sm = 0;
      const cudaError_t e = pass_shape(h, ax, base, jobs.size(), -1, P, thr, sm);
      if (e != cudaSuccess) return e;
      const int var = (P.KP == 3 ? 2 : 0) + (P.ff ? 1 : 0);
      const long long nbx = (P.nlines + P.L - 1) / P.L;
      if (nbx * STAB_MAX_JOBS > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
      for (size_t j0 = 0; j0 < jobs.size(); j0 += STAB_MAX_JOBS) {
        P.njobs = (int)std::min<size_t>(STAB_MAX_JOBS, jobs.size() - j0);
        for (int k = 0; k < P.njobs; ++k) P.job[k] = jobs[j0 + k];
        items[var].push_back(P);
        blocks[var].push_back((int)(nbx * P.njobs));
      }
      threads[var] = std::max(threads[var], thr);
      smem[var] = std::max(smem[var], sm);
    }
    for (int k = 0; k < 4; ++k) plan.line[q][k] = im.section(items[k], blocks[k], threads[k], smem[k]);
  }
  for (int d = 0; d < 2; ++d) plan.point[d] = im.section(points[d], point_blocks[d], 128, 0);
  return im.overflow ? cudaErrorInvalidValue : cudaSuccess;
}

// The launches of a planned batched J v; d = device copy of the image.
cudaError_t jv_batch_launch(const JvBatchPlan& plan, const unsigned char* d, cudaStream_t st) {
  auto items_of = [&](const BatchSection& s) { return (const void*)(d + s.items); };
  auto start_of = [&](const BatchSection& s) { return (const int*)(d + s.start); };
  if (plan.norm.count)
    k_norm2_batch<<<plan.norm.blocks, 256, 0, st>>>((const NormItem*)items_of(plan.norm), start_of(plan.norm),
                                                    plan.norm.count);
  if (plan.temp.count)
    k_temperature_fast_batch<<<plan.temp.blocks, 128, 0, st>>>((const TempItem*)items_of(plan.temp),
                                                               start_of(plan.temp), plan.temp.count);
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < 4; ++k) {
      const BatchSection& s = plan.line[q][k];
      if (!s.count) continue;
      const PassParams* it = (const PassParams*)items_of(s);
      if (k == 0) k_line_pass_batch<false><<<s.blocks, s.threads, s.smem, st>>>(it, start_of(s), s.count);
      else if (k == 1) k_line_pass_batch<true><<<s.blocks, s.threads, s.smem, st>>>(it, start_of(s), s.count);
      else if (k == 2) k_line_pass_compact_batch<false><<<s.blocks, s.threads, s.smem, st>>>(it, start_of(s), s.count);
      else k_line_pass_compact_batch<true><<<s.blocks, s.threads, s.smem, st>>>(it, start_of(s), s.count);
    }
  if (plan.point[0].count)
    k_point_fast_batch<2><<<plan.point[0].blocks, 128, 0, st>>>((const PointItem*)items_of(plan.point[0]),
                                                               start_of(plan.point[0]), plan.point[0].count);
  if (plan.point[1].count)
    k_point_fast_batch<3><<<plan.point[1].blocks, 128, 0, st>>>((const PointItem*)items_of(plan.point[1]),
                                                               start_of(plan.point[1]), plan.point[1].count);
  return cudaGetLastError();
}

// Batched ||v|| (mode 1) or ||v||^2 (mode 0): each job with its handle's
// reduction partials and block count, so each result equals launch_norm2's.
cudaError_t norm_batch_plan(const std::vector<NormJob>& jobs, BatchImage& im, BatchSection& sec) {
  std::vector<NormItem> items;
  std::vector<int> blocks;
  for (const NormJob& J : jobs) {
    StabHandle* h = J.h;
    long long nb = (J.n + 1023) / 1024;
    nb = std::max<long long>(1, std::min<long long>(nb, h->red_blocks));
    NormItem it{};
    it.v = J.v;
    it.n = J.n;
    it.partial = h->d_red;
    it.counter = (unsigned*)(h->d_red + h->red_blocks + 8);
    it.out = J.out;
    it.q0norm = h->q0norm;
    it.fixed_eps = h->opts.eps;
    it.mode = J.mode;
    it.gate = J.gate;
    items.push_back(it);
    blocks.push_back((int)nb);
  }
  sec = im.section(items, blocks, 256, 0);
  return im.overflow ? cudaErrorInvalidValue : cudaSuccess;
}

cudaError_t norm_batch_launch(const BatchSection& sec, const unsigned char* d, cudaStream_t st) {
  if (!sec.count) return cudaSuccess;
  k_norm2_batch<<<sec.blocks, 256, 0, st>>>((const NormItem*)(d + sec.items), (const int*)(d + sec.start), sec.count);
  return cudaGetLastError();
}

// Epsilon of the exact-tangent instances is zero (set once before their J v).
cudaError_t jv_batch_zero_eps(const JvBatchPlan& plan, cudaStream_t st) {
  for (double* e : plan.zero_eps) k_set_scalar<<<1, 1, 0, st>>>(e, 0.0);
  return cudaGetLastError();
}

static cudaError_t jv_batch_apply(stab_jv_batch_s* B, const double2* const* v, double2* const* out, const double* shifts) {
  BatchImage im;
  JvBatchPlan plan;
  std::vector<double2> sh;
  if (shifts)
    for (size_t i = 0; i < B->hs.size(); ++i) sh.push_back(make_double2(shifts[2 * i], shifts[2 * i + 1]));
  cudaError_t e = jv_batch_plan(B->hs, v, out, shifts ? sh.data() : nullptr, nullptr, im, plan);
  if (e != cudaSuccess) return e;
  if ((e = batch_stage(B, im)) != cudaSuccess) return e;
  if ((e = batch_order_begin(B)) != cudaSuccess) return e;
  // exact tangent: epsilon is zero
  for (StabHandle* h : B->hs)
    if (h->opts.eps_mode == 2 && h->last_eps_mode != 2) k_set_scalar<<<1, 1, 0, B->stream>>>(h->d_eps, 0.0);
  if ((e = jv_batch_launch(plan, (const unsigned char*)B->d_buf, B->stream)) != cudaSuccess) return e;
  for (StabHandle* h : B->hs) {
    h->last_eps_mode = h->opts.eps_mode;
    h->stats.jv_calls++;
  }
  return batch_order_end(B);
}

extern "C" stab_status stab_jv_batch_create(stab_jv_batch* out, const stab_handle* handles, int count, void* cuda_stream) {
  if (!out) return STAB_ERR_INVALID_ARG;
  *out = nullptr;
  if (!handles || count < 1 || count > 4096) return STAB_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return STAB_ERR_CUDA;
  std::vector<StabHandle*> hs((size_t)count);
  for (int i = 0; i < count; ++i) hs[i] = (StabHandle*)handles[i];  // the handle type derives from StabHandle
  for (int i = 0; i < count; ++i) {
    StabHandle* h = hs[i];
    if (!h || h->device != dev) return STAB_ERR_INVALID_ARG;
    for (int k = 0; k < i; ++k)
      if (hs[k] == h) return STAB_ERR_INVALID_ARG;  // one derivative scratch per handle
    if (!(h->homog && h->d_coef && !h->force_dn_path)) return STAB_ERR_UNSUPPORTED;
  }
  stab_jv_batch_s* B = new (std::nothrow) stab_jv_batch_s();
  if (!B) return STAB_ERR_OOM;
  B->hs = hs;
  B->device = dev;
  B->stream = (cudaStream_t)cuda_stream;
  if (jv_batch_attributes() != cudaSuccess ||
      cudaEventCreateWithFlags(&B->copied, cudaEventDisableTiming) != cudaSuccess) {
    delete B;
    return STAB_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&B->order, cudaEventDisableTiming) != cudaSuccess) {
    cudaEventDestroy(B->copied);
    delete B;
    return STAB_ERR_CUDA;
  }
  *out = B;
  return STAB_OK;
}

extern "C" stab_status stab_jv_batch_apply(stab_jv_batch B, const void* const* v, void* const* Jv, const double* shifts) {
  if (!B) return STAB_ERR_INVALID_ARG;
  if (!v || !Jv) {
    B->err = "stab_jv_batch_apply: null vector list";
    return STAB_ERR_INVALID_ARG;
  }
  const int count = (int)B->hs.size();
  for (int i = 0; i < count; ++i) {
    const char* a = (const char*)v[i];
    const char* b = (const char*)Jv[i];
    const long long bytes = B->hs[i]->n * (long long)sizeof(double2);
    if (!a || !b || (a < b + bytes && b < a + bytes)) {
      B->err = "stab_jv_batch_apply: null or overlapping v / Jv of instance " + std::to_string(i);
      return STAB_ERR_INVALID_ARG;
    }
  }
  const cudaError_t e = jv_batch_apply(B, (const double2* const*)v, (double2* const*)Jv, shifts);
  if (e != cudaSuccess) {
    B->err = std::string("stab_jv_batch_apply: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA;
  }
  return STAB_OK;
}

extern "C" const char* stab_jv_batch_last_error(stab_jv_batch B) { return B ? B->err.c_str() : ""; }

extern "C" void stab_jv_batch_destroy(stab_jv_batch B) {
  if (!B) return;
  // the batch's kernels read the handles' scratch, tables and inverses: wait
  // for all of them before the handles may be destroyed
  cudaStreamSynchronize(B->stream);
  cudaEventSynchronize(B->copied);
  if (B->d_buf) cudaFreeAsync(B->d_buf, B->stream);
  if (B->h_buf) cudaFreeHost(B->h_buf);
  cudaEventDestroy(B->copied);
  if (B->order) cudaEventDestroy(B->order);
  delete B;
}
