// Local block-Jacobi preconditioner (Sec. "Preconditioning"): one dense
// block per tile of tx x ty (x tz) grid points with all variables, equal to
// the principal submatrix of (J - sigma I) over the tile's unknowns, J the
// exact tangent.  The block is assembled from the linearised pointwise
// operator fed with unit perturbations: a perturbation at tile point q only
// reaches tile point p through the entries of the dense 1-D derivative
// matrices (A^{-1} B of the compact schemes) that couple q and p, so the
// restriction to the tile is exact.  Blocks are inverted by Gauss-Jordan
// elimination with partial pivoting (first row of maximum modulus) and
// applied as a batched block matrix-vector product.
// Local unknown order inside a tile: [var][lz][ly][lx], lx fastest.
#include <cublas_v2.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "pointwise.cuh"

pw::Phys phys_of(const StabHandle* h);

namespace {

struct AsmParams {
  int nx, ny, nz, tx, ty, tz, ntx, nty, ntpts, bsz;
  long long npts, nbase, tile0;
  int homog;
  const double* btab;
  const double* eta_y;
  const double* eta_yy;
  const unsigned char* bcflags;
  const double2* Dm1[3];  // [l * n + t] = (D e_l)_t: first-derivative matrix of axis a, column-major
  const double2* Dm2[3];
  int nax[3];
  pw::Phys phys;
  double2 sigma;
  double2* out;  // [tile - tile0][row][col]
};

// Column (beta, q) of the linearised operator at the rows of point p (all
// variables), for grid points p and q that lie in the same tile: the unit
// perturbation's derivatives come from the 1-D derivative matrices, the
// coefficients from the base table.
template <int D>
__device__ __forceinline__ void asm_entry(const AsmParams& P, const int gp[3], const int gq[3], int beta,
                                          double res[D + 2]) {
  const long long ptp = ((long long)gp[2] * P.ny + gp[1]) * P.nx + gp[0];
  const long long ptq = ((long long)gq[2] * P.ny + gq[1]) * P.nx + gq[0];
  const long long bp = P.homog ? gp[1] : ptp, bq = P.homog ? gq[1] : ptq;
  const double ig = P.phys.C.ig;
  // field values at q of the unit perturbation (fields 0..D+1 = variables, D+2 = T)
  double fq[D + 3];
#pragma unroll
  for (int f = 0; f < D + 2; ++f) fq[f] = f == beta ? 1.0 : 0.0;
  {
    const double T0 = P.btab[(long long)pw::bt_val(D, D + 2) * P.nbase + bq];
    const double ip0 = P.btab[(long long)pw::bt_extra(D, pw::X_IP) * P.nbase + bq];
    fq[D + 2] = beta == 0 ? T0 * (1.0 - ig) * ip0 : (beta == D + 1 ? T0 * P.phys.C.icp : 0.0);
  }
  const double ey = P.eta_y[gp[1]], eyy = P.eta_yy[gp[1]];
  bool same[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) same[a] = gp[a] == gq[a];
  auto d1c = [&](int a) { return P.Dm1[a][(long long)gq[a] * P.nax[a] + gp[a]].x; };  // D[p][q]
  auto d2c = [&](int a) { return P.Dm2[a][(long long)gq[a] * P.nax[a] + gp[a]].x; };
  pw::WIn<D> W;
  const bool at_q = same[0] && same[1] && same[2];
#pragma unroll
  for (int f = 0; f < D + 3; ++f) W.v[f] = at_q ? fq[f] : 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    bool line = true;  // p and q differ only along axis a
#pragma unroll
    for (int c = 0; c < 3; ++c)
      if (c != a && !same[c]) line = false;
    const double c1 = line ? d1c(a) * (a == 1 ? ey : 1.0) : 0.0;
    double c2 = 0.0;
    if (line) c2 = a == 1 ? fma(d2c(a), ey * ey, d1c(a) * eyy) : d2c(a);
#pragma unroll
    for (int f = 0; f < D + 3; ++f) W.d1[a][f] = c1 * fq[f];
#pragma unroll
    for (int g = 0; g < D + 1; ++g) W.d2[a][g] = c2 * fq[g < D ? 1 + g : D + 2];
  }
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      double w = 0.0;
      if (a != c) {
        bool plane = true;  // p and q differ only along axes a and c
#pragma unroll
        for (int o = 0; o < 3; ++o)
          if (o != a && o != c && !same[o]) plane = false;
        if (plane) w = d1c(a) * d1c(c) * ((a == 1 || c == 1) ? ey : 1.0) * fq[1 + c];
      }
      W.mix[a][c] = w;
    }
  auto B = [&](int slot) { return P.btab[(long long)slot * P.nbase + bp]; };
  const bool bc_row = gp[1] == 0 || gp[1] == P.ny - 1;
  const unsigned fl =
      bc_row ? P.bcflags[(gp[1] == P.ny - 1 ? (long long)P.nx * P.nz : 0) + (long long)gp[2] * P.nx + gp[0]] : 0u;
  pw::rhs_diff<D>(P.phys, B, W, 0.0, bc_row, fl, res);
}

template <int D>
__global__ void __launch_bounds__(128) k_assemble(const AsmParams P) {
  const long long tile = P.tile0 + blockIdx.x;
  const int tX = (int)(tile % P.ntx);
  const int tY = (int)((tile / P.ntx) % P.nty);
  const int tZ = (int)(tile / ((long long)P.ntx * P.nty));
  const int x0 = tX * P.tx, y0 = tY * P.ty, z0 = tZ * P.tz;
  const int T = P.ntpts, bsz = P.bsz;
  double2* blk = P.out + (long long)blockIdx.x * bsz * bsz;
  for (long long idx = threadIdx.x; idx < (long long)bsz * T; idx += blockDim.x) {
    const int col = (int)(idx / T), pp = (int)(idx % T);
    const int beta = col / T, q = col % T;
    const int qx = q % P.tx, qy = (q / P.tx) % P.ty, qz = q / (P.tx * P.ty);
    const int px = pp % P.tx, py = (pp / P.tx) % P.ty, pz = pp / (P.tx * P.ty);
    const int gq[3] = {x0 + qx, y0 + qy, z0 + qz};
    const int gp[3] = {x0 + px, y0 + py, z0 + pz};
    double res[D + 2];
    asm_entry<D>(P, gp, gq, beta, res);
#pragma unroll
    for (int a = 0; a < D + 2; ++a) {
      const int row = a * T + pp;
      double2 val = make_double2(res[a], 0.0);
      if (row == col) { val.x -= P.sigma.x; val.y -= P.sigma.y; }
      blk[(long long)row * bsz + col] = val;
    }
  }
}

// Reduced-operator tiles in block-tridiagonal form.  A tile's points are
// grouped in levels of two y lines (level l: local y in {2l, 2l + 1}); with
// the three-point interior stencils and the end rows reaching three points in,
// a level couples only to itself and its two neighbours.  Level unknowns are
// ordered [var][lz][ly][lx] (m = nv * 2 * tx * tz).  Grid (tiles, levels, 3):
// kind 0 = L_l (columns of level l - 1), 1 = D_l (- sigma on the diagonal),
// 2 = U_l (columns of level l + 1); out[tile][l][kind] is m x m, row-major.
template <int D>
__global__ void __launch_bounds__(128) k_assemble_bt(const AsmParams P, int m, int nlev, double2* out) {
  const int lev = blockIdx.y, kind = blockIdx.z;
  const int ql = lev + kind - 1;
  if (ql < 0 || ql >= nlev) return;
  const long long tile = P.tile0 + blockIdx.x;
  const int tX = (int)(tile % P.ntx);
  const int tY = (int)((tile / P.ntx) % P.nty);
  const int tZ = (int)(tile / ((long long)P.ntx * P.nty));
  const int x0 = tX * P.tx, y0 = tY * P.ty, z0 = tZ * P.tz;
  const int NP = 2 * P.tx * P.tz;
  double2* blk = out + (((long long)blockIdx.x * nlev + lev) * 3 + kind) * m * m;
  for (int idx = threadIdx.x; idx < m * NP; idx += blockDim.x) {
    const int col = idx / NP, pp = idx % NP;
    const int beta = col / NP, q = col % NP;
    const int gq[3] = {x0 + q % P.tx, y0 + 2 * ql + (q / P.tx) % 2, z0 + q / (2 * P.tx)};
    const int gp[3] = {x0 + pp % P.tx, y0 + 2 * lev + (pp / P.tx) % 2, z0 + pp / (2 * P.tx)};
    double res[D + 2];
    asm_entry<D>(P, gp, gq, beta, res);
#pragma unroll
    for (int a = 0; a < D + 2; ++a) {
      const int row = a * NP + pp;
      double2 val = make_double2(res[a], 0.0);
      if (kind == 1 && row == col) { val.x -= P.sigma.x; val.y -= P.sigma.y; }
      blk[(long long)row * m + col] = val;
    }
  }
}

template <class R>
struct C2 {
  R x, y;
};

__global__ void k_to_float(const double2* in, float2* out, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    double2 v = in[i];
    out[i] = make_float2((float)v.x, (float)v.y);
  }
}

// In-place Gauss-Jordan inversion with partial pivoting of one b x b complex
// block per CTA (row-major).  Threads own columns; rows are swept in order.
// The sweep of one block M (b x b, row-major) by the calling CTA; prow, pcol:
// b complex, perm: b ints, in shared memory.  Returns (thread 0) the first
// step whose pivot column was zero, plus one, else 0.
template <class R>
__device__ int gj_sweep(C2<R>* M, int b, C2<R>* prow, C2<R>* pcol, int* perm) {
  __shared__ double rv[32];
  __shared__ int ri[32];
  __shared__ int s_piv;
  const int nthr = blockDim.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int bad = 0;
  for (int k = 0; k < b; ++k) {
    // pivot: first row i >= k of maximum |A[i][k]|
    double best = -1.0;
    int bi = b;
    for (int i = k + threadIdx.x; i < b; i += nthr) {
      C2<R> v = M[(long long)i * b + k];
      double m = (double)v.x * v.x + (double)v.y * v.y;
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = -1.0;
      int bbi = b;
      for (int w = 0; w < (nthr + 31) / 32; ++w)
        if (rv[w] > bb || (rv[w] == bb && ri[w] < bbi)) { bb = rv[w]; bbi = ri[w]; }
      if (!(bb > 0.0)) { bad = k + 1; bbi = k; }
      s_piv = bbi;
      perm[k] = bbi;
    }
    __syncthreads();
    const int p = s_piv;
    for (int j = threadIdx.x; j < b; j += nthr) {
      C2<R> a = M[(long long)k * b + j], c = M[(long long)p * b + j];
      if (p != k) { M[(long long)k * b + j] = c; M[(long long)p * b + j] = a; }
      prow[j] = p != k ? c : a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < b; i += nthr) pcol[i] = M[(long long)i * b + k];
    __syncthreads();
    C2<R> pv = prow[k];
    R den = pv.x * pv.x + pv.y * pv.y;
    if (!(den > (R)0)) den = (R)1;
    const C2<R> inv = {pv.x / den, -pv.y / den};
    for (int j = threadIdx.x; j < b; j += nthr) {
      const C2<R> pj = prow[j];
      const C2<R> s = {pj.x * inv.x - pj.y * inv.y, pj.x * inv.y + pj.y * inv.x};  // prow[j] / pivot
      C2<R>* col = M + j;
      if (j == k) {  // the pivot column: -pcol / pivot, and 1 / pivot on the diagonal
        for (int i = 0; i < b; ++i) {
          const C2<R> ci = pcol[i];
          col[(long long)i * b] = i == k ? inv : C2<R>{-(ci.x * inv.x - ci.y * inv.y), -(ci.x * inv.y + ci.y * inv.x)};
        }
        continue;
      }
      // rows in groups of 8: all loads first, so eight L2 round trips are in flight per thread
      constexpr int G = 8;
      for (int i0 = 0; i0 < b; i0 += G) {
        C2<R> v[G];
#pragma unroll
        for (int q = 0; q < G; ++q)
          if (i0 + q < b) v[q] = col[(long long)(i0 + q) * b];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int i = i0 + q;
          if (i >= b) break;
          const C2<R> ci = pcol[i];
          if (i == k) {
            v[q] = s;
          } else {
            v[q].x -= ci.x * s.x - ci.y * s.y;
            v[q].y -= ci.x * s.y + ci.y * s.x;
          }
          col[(long long)i * b] = v[q];
        }
      }
    }
    __syncthreads();
  }
  // undo the row interchanges: swap columns in reverse order
  for (int k = b - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = threadIdx.x; i < b; i += nthr) {
        C2<R> t = M[(long long)i * b + k];
        M[(long long)i * b + k] = M[(long long)i * b + p];
        M[(long long)i * b + p] = t;
      }
    __syncthreads();
  }
  return bad;
}

template <class R>
__global__ void k_gauss_jordan(C2<R>* A, int b, int* info) {
  extern __shared__ unsigned char smraw[];
  C2<R>* prow = (C2<R>*)smraw;
  C2<R>* pcol = prow + b;
  int* perm = (int*)(pcol + b);
  const int bad = gj_sweep<R>(A + (long long)blockIdx.x * b * b, b, prow, pcol, perm);
  if (threadIdx.x == 0 && bad) atomicMax(info, 1);
}

// Block-tridiagonal LU of a reduced-operator tile (one CTA per tile, levels in
// order; block Thomas elimination): S_0 = D_0, S_l = D_l - L_l X_{l-1},
// X_l = S_l^{-1} U_l, with S_l inverted by the Gauss-Jordan sweep above
// (partial pivoting inside the level).  Stored per level
// F[tile][l] = {P_l = S_l^{-1} L_l, S_l^{-1}, X_l}: the forward substitution
// y_l = S_l^{-1} (q_l - L_l y_{l-1}) = S_l^{-1} q_l - P_l y_{l-1} then has one
// product per level on its dependency chain, and the S_l^{-1} q_l of all
// levels are independent.
template <class R>
__global__ void k_bt_factor(const double2* asmb, C2<R>* F, int m, int nlev, int* info) {
  extern __shared__ unsigned char smraw[];
  C2<R>* prow = (C2<R>*)smraw;
  C2<R>* pcol = prow + m;
  int* perm = (int*)(pcol + m);
  const long long mm = (long long)m * m;
  const double2* A = asmb + (long long)blockIdx.x * nlev * 3 * mm;
  C2<R>* Ft = F + (long long)blockIdx.x * nlev * 3 * mm;
  int bad = 0;
  for (int l = 0; l < nlev; ++l) {
    const double2* Al = A + (long long)l * 3 * mm;
    C2<R>* Pl = Ft + (long long)l * 3 * mm;
    C2<R>* S = Pl + mm;
    C2<R>* X = S + mm;
    const C2<R>* Xp = Pl - mm;  // X_{l-1}
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const double2 dv = Al[mm + idx];
      C2<R> sv = {(R)dv.x, (R)dv.y};
      if (l > 0) {
        const int i = idx / m, c = idx - (idx / m) * m;
        R ax = 0, ay = 0;
        for (int k = 0; k < m; ++k) {
          const double2 a = Al[(long long)i * m + k];
          const C2<R> x = Xp[(long long)k * m + c];
          ax += (R)a.x * x.x - (R)a.y * x.y;
          ay += (R)a.x * x.y + (R)a.y * x.x;
        }
        sv.x -= ax;
        sv.y -= ay;
      }
      S[idx] = sv;
    }
    __syncthreads();
    const int b = gj_sweep<R>(S, m, prow, pcol, perm);
    if (b && !bad) bad = b;
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = idx / m, c = idx - (idx / m) * m;
      R px = 0, py = 0, xx = 0, xy = 0;
      for (int k = 0; k < m; ++k) {
        const C2<R> a = S[(long long)i * m + k];
        if (l > 0) {
          const double2 lv = Al[(long long)k * m + c];
          px += a.x * (R)lv.x - a.y * (R)lv.y;
          py += a.x * (R)lv.y + a.y * (R)lv.x;
        }
        if (l + 1 < nlev) {
          const double2 u = Al[2 * mm + (long long)k * m + c];
          xx += a.x * (R)u.x - a.y * (R)u.y;
          xy += a.x * (R)u.y + a.y * (R)u.x;
        }
      }
      Pl[idx] = C2<R>{px, py};
      X[idx] = C2<R>{xx, xy};
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicMax(info, 1);
}

struct BtApplyParams {
  const double2* q;
  const float2* q32;  // FP32 input (GMRES with an FP32 basis) instead of q
  double2* z;
  const void* F;
  int m, nlev, tx, ty, tz, ntx, nty, nx, ny;
  long long npts;
  const int* gate;
};

__device__ __forceinline__ long long bt_dof(const BtApplyParams& P, long long tile, int l, int r) {
  const int NP = 2 * P.tx * P.tz;
  const int tX = (int)(tile % P.ntx), tY = (int)((tile / P.ntx) % P.nty), tZ = (int)(tile / ((long long)P.ntx * P.nty));
  const int a = r / NP, pp = r % NP;
  const int x = tX * P.tx + pp % P.tx, y = tY * P.ty + 2 * l + (pp / P.tx) % 2, z = tZ * P.tz + pp / (2 * P.tx);
  return (long long)a * P.npts + ((long long)z * P.ny + y) * P.nx + x;
}

// Rows per CTA and threads per row of the level products: G threads (a power
// of two) share a row, G * m <= blockDim.
__device__ __forceinline__ int bt_group(int m) {
  int G = 1;
  while (G < 32 && 2 * G * m <= (int)blockDim.x) G *= 2;
  return G;
}

// w_l = S_l^{-1} q_l for every level of every tile, into z (grid: tiles x levels).
// KP > 0: each thread's row fragment (at most KP entries) is loaded in one
// unrolled batch, so all its loads are in flight together.
template <class R, bool Q32, int KP>
__global__ void __launch_bounds__(256) k_bt_rhs(const BtApplyParams P) {
  if (P.gate && *P.gate) return;
  extern __shared__ unsigned char smraw[];
  C2<R>* t = (C2<R>*)smraw;
  const int m = P.m, l = blockIdx.y;
  const long long tile = blockIdx.x, mm = (long long)m * m;
  const C2<R>* S = (const C2<R>*)P.F + (tile * P.nlev + l) * 3 * mm + mm;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const long long d = bt_dof(P, tile, l, r);
    if (Q32) { const float2 v = P.q32[d]; t[r] = C2<R>{(R)v.x, (R)v.y}; }
    else { const double2 v = P.q[d]; t[r] = C2<R>{(R)v.x, (R)v.y}; }
  }
  __syncthreads();
  const int G = bt_group(m);
  const int row = threadIdx.x / G, g = threadIdx.x % G;
  R sx = 0, sy = 0;
  if (KP > 0) {
    C2<R> a[KP > 0 ? KP : 1];
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k = g + j * G;
      a[j] = (row < m && k < m) ? S[(long long)row * m + k] : C2<R>{0, 0};
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k = g + j * G;
      const C2<R> b = k < m ? t[k] : C2<R>{0, 0};
      sx += a[j].x * b.x - a[j].y * b.y;
      sy += a[j].x * b.y + a[j].y * b.x;
    }
  } else if (row < m) {
    for (int k = g; k < m; k += G) {
      const C2<R> a = S[(long long)row * m + k], b = t[k];
      sx += a.x * b.x - a.y * b.y;
      sy += a.x * b.y + a.y * b.x;
    }
  }
  for (int o = G >> 1; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  if (row < m && g == 0) P.z[bt_dof(P, tile, l, row)] = make_double2((double)sx, (double)sy);
}

// The level recurrences of one tile (one CTA per tile), z holding w on entry:
// forward y_l = w_l - P_l y_{l-1}, backward x_l = y_l - X_l x_{l+1}.  Each row's
// product is split over G threads; with KP > 0 every thread holds its
// fragment (at most KP entries) of the next level's matrix and the next w in
// registers, loaded while the current level is reduced, so the dependency
// chain carries no global-memory latency.
template <class R, int KP>
__global__ void __launch_bounds__(256) k_bt_sweep(const BtApplyParams P) {
  if (P.gate && *P.gate) return;
  extern __shared__ unsigned char smraw[];
  C2<R>* va = (C2<R>*)smraw;
  C2<R>* vb = va + P.m;
  const int m = P.m, nlev = P.nlev;
  const long long tile = blockIdx.x, mm = (long long)m * m;
  const C2<R>* Ft = (const C2<R>*)P.F + tile * nlev * 3 * mm;
  const int G = bt_group(m);
  const int row = threadIdx.x / G, g = threadIdx.x % G;
  const bool act = row < m, lead = act && g == 0;
  C2<R> cur[KP > 0 ? KP : 1], nxt[KP > 0 ? KP : 1];
  auto fetch = [&](C2<R>* frag, const C2<R>* M) {
#pragma unroll
    for (int j = 0; j < KP; ++j) {
      const int k = g + j * G;
      frag[j] = (act && k < m) ? M[(long long)row * m + k] : C2<R>{0, 0};
    }
  };
  // (M x)_row from registers (KP > 0) or from memory, complete in every lane of the row's group
  auto mv = [&](const C2<R>* frag, const C2<R>* M, const C2<R>* x) {
    R sx = 0, sy = 0;
    if (KP > 0) {
#pragma unroll
      for (int j = 0; j < KP; ++j) {
        const int k = g + j * G;
        const C2<R> b = k < m ? x[k] : C2<R>{0, 0};
        sx += frag[j].x * b.x - frag[j].y * b.y;
        sy += frag[j].x * b.y + frag[j].y * b.x;
      }
    } else if (act) {
      for (int k = g; k < m; k += G) {
        const C2<R> a = M[(long long)row * m + k], b = x[k];
        sx += a.x * b.x - a.y * b.y;
        sy += a.x * b.y + a.y * b.x;
      }
    }
    for (int o = G >> 1; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    return C2<R>{sx, sy};
  };
  // forward: y_0 = w_0
  C2<R>* yp = va;
  C2<R>* yc = vb;
  double2 wn = make_double2(0.0, 0.0);
  if (lead) {
    const double2 w = P.z[bt_dof(P, tile, 0, row)];
    yp[row] = C2<R>{(R)w.x, (R)w.y};
    if (nlev > 1) wn = P.z[bt_dof(P, tile, 1, row)];
  }
  if (KP > 0 && nlev > 1) fetch(nxt, Ft + 3 * mm);
  __syncthreads();
  for (int l = 1; l < nlev; ++l) {
    const C2<R>* Pl = Ft + (long long)l * 3 * mm;
    const double2 w = wn;
    if (KP > 0) {
#pragma unroll
      for (int j = 0; j < KP; ++j) cur[j] = nxt[j];
      if (l + 1 < nlev) fetch(nxt, Pl + 3 * mm);
    }
    if (lead && l + 1 < nlev) wn = P.z[bt_dof(P, tile, l + 1, row)];
    const C2<R> s = mv(cur, Pl, yp);
    if (lead) {
      const C2<R> y = {(R)w.x - s.x, (R)w.y - s.y};
      yc[row] = y;
      P.z[bt_dof(P, tile, l, row)] = make_double2((double)y.x, (double)y.y);
    }
    __syncthreads();
    C2<R>* tmp = yp; yp = yc; yc = tmp;
  }
  // backward: x_{nlev-1} = y_{nlev-1} (in yp)
  if (KP > 0 && nlev > 1) fetch(nxt, Ft + (long long)(nlev - 2) * 3 * mm + 2 * mm);
  double2 yn = make_double2(0.0, 0.0);
  if (lead && nlev > 1) yn = P.z[bt_dof(P, tile, nlev - 2, row)];
  for (int l = nlev - 2; l >= 0; --l) {
    const C2<R>* Xl = Ft + (long long)l * 3 * mm + 2 * mm;
    const double2 y = yn;
    if (KP > 0) {
#pragma unroll
      for (int j = 0; j < KP; ++j) cur[j] = nxt[j];
      if (l > 0) fetch(nxt, Xl - 3 * mm);
    }
    if (lead && l > 0) yn = P.z[bt_dof(P, tile, l - 1, row)];
    const C2<R> s = mv(cur, Xl, yp);
    if (lead) {
      const C2<R> x = {(R)y.x - s.x, (R)y.y - s.y};
      yc[row] = x;
      P.z[bt_dof(P, tile, l, row)] = make_double2((double)x.x, (double)x.y);
    }
    __syncthreads();
    C2<R>* tmp = yp; yp = yc; yc = tmp;
  }
}

struct ApplyParams {
  const double2* q;
  double2* z;
  const void* inv;
  int nx, ny, tx, ty, tz, ntx, nty, ntpts, bsz;
  long long npts;
  const int* gate;  // when set and nonzero the launch does nothing (graph-captured GMRES after convergence)
  const float2* q32;  // FP32 input (GMRES with an FP32 basis) instead of q
};

__device__ __forceinline__ long long tile_dof(const ApplyParams& P, long long tile, int r) {
  const int tX = (int)(tile % P.ntx), tY = (int)((tile / P.ntx) % P.nty), tZ = (int)(tile / ((long long)P.ntx * P.nty));
  const int var = r / P.ntpts, pp = r % P.ntpts;
  const int px = pp % P.tx, py = (pp / P.tx) % P.ty, pz = pp / (P.tx * P.ty);
  return (long long)var * P.npts + ((long long)(tZ * P.tz + pz) * P.ny + (tY * P.ty + py)) * P.nx + tX * P.tx + px;
}

// z_tile = Minv_tile q_tile with the inverse stored column-major (BF16
// storage: Mt[c * b + r] = Minv[r][c]).  Grid (tiles, row slices); a CTA stages its
// tile of q in shared memory and each thread forms one row: every load is a
// coalesced segment of a column, eight loads in flight per thread, no
// reductions.  S: stored complex type, R: accumulation type.
template <class S, class R>
__device__ __forceinline__ void load_c(const S* p, R& x, R& y);
template <>
__device__ __forceinline__ void load_c<__nv_bfloat162, float>(const __nv_bfloat162* p, float& x, float& y) {
  const float2 v = __bfloat1622float2(__ldg(p));
  x = v.x;
  y = v.y;
}

// one CTA: row slice `slice` of `nslices` of tile `tile`
template <class S, class R, bool Q32>
__device__ __forceinline__ void apply_cols_body(const ApplyParams& P, long long tile, unsigned slice, unsigned nslices) {
  extern __shared__ unsigned char smraw[];
  C2<R>* qs = (C2<R>*)smraw;
  const int b = P.bsz;
  const int rb0 = (int)((long long)b * slice / nslices);
  const int rb1 = (int)((long long)b * (slice + 1) / nslices);
  const S* Mt = (const S*)P.inv + (long long)tile * b * b;
  for (int r = threadIdx.x; r < b; r += blockDim.x) {
    const long long d = tile_dof(P, tile, r);
    if (Q32) {
      const float2 v = P.q32[d];
      qs[r] = C2<R>{(R)v.x, (R)v.y};
    } else {
      const double2 v = P.q[d];
      qs[r] = C2<R>{(R)v.x, (R)v.y};
    }
  }
  __syncthreads();
  for (int r = rb0 + threadIdx.x; r < rb1; r += blockDim.x) {
    const S* col = Mt + r;
    R ar = 0, ai = 0;
#pragma unroll 8
    for (int c = 0; c < b; ++c) {
      R mx, my;
      load_c<S, R>(col + (long long)c * b, mx, my);
      const C2<R> x = qs[c];
      ar += mx * x.x - my * x.y;
      ai += mx * x.y + my * x.x;
    }
    P.z[tile_dof(P, tile, r)] = make_double2((double)ar, (double)ai);
  }
}

template <class S, class R, bool Q32>
__global__ void k_apply_cols(const ApplyParams P) {
  if (P.gate && *P.gate) return;
  apply_cols_body<S, R, Q32>(P, blockIdx.x, blockIdx.y, gridDim.y);
}

// The same product for blocks of a multiple of four rows: each thread forms
// four consecutive rows from one 16-byte load per column (four BF16 complex
// entries), so a warp moves 512 bytes per load instruction.
template <bool Q32>
__device__ __forceinline__ void apply_cols4_body(const ApplyParams& P, long long tile, unsigned slice, unsigned nslices) {
  extern __shared__ unsigned char smraw[];
  float2* qs = (float2*)smraw;
  const int b = P.bsz, b4 = P.bsz >> 2;
  const int q0 = (int)((long long)b4 * slice / nslices);
  const int q1 = (int)((long long)b4 * (slice + 1) / nslices);
  const uint4* Mt = (const uint4*)((const __nv_bfloat162*)P.inv + (long long)tile * b * b);
  for (int r = threadIdx.x; r < b; r += blockDim.x) {
    const long long d = tile_dof(P, tile, r);
    if (Q32) {
      qs[r] = P.q32[d];
    } else {
      const double2 v = P.q[d];
      qs[r] = make_float2((float)v.x, (float)v.y);
    }
  }
  __syncthreads();
  for (int r4 = q0 + threadIdx.x; r4 < q1; r4 += blockDim.x) {
    const uint4* col = Mt + r4;
    float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int c = 0; c < b; ++c) {
      const uint4 u = __ldg(col + (long long)c * b4);
      const float2 x = qs[c];
      const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        __nv_bfloat162 e;
        memcpy(&e, &w[k], sizeof(e));
        const float2 m = __bfloat1622float2(e);
        ar[k] += m.x * x.x - m.y * x.y;
        ai[k] += m.x * x.y + m.y * x.x;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) P.z[tile_dof(P, tile, 4 * r4 + k)] = make_double2((double)ar[k], (double)ai[k]);
  }
}

template <bool Q32>
__global__ void k_apply_cols4(const ApplyParams P) {
  if (P.gate && *P.gate) return;
  apply_cols4_body<Q32>(P, blockIdx.x, blockIdx.y, gridDim.y);
}

// z_tile = Minv_tile q_tile with the inverse stored row-major (FP64 or FP32):
// one warp per row at a time, FP32 rows of even length read two entries per
// 16-byte load; grid (tiles, row slices) as above.
template <class R, bool Q32>
__device__ __forceinline__ void apply_rows_body(const ApplyParams& P, long long tile, unsigned slice, unsigned nslices) {
  extern __shared__ unsigned char smraw[];
  C2<R>* qs = (C2<R>*)smraw;
  const int rb0 = (int)((long long)P.bsz * slice / nslices);
  const int rb1 = (int)((long long)P.bsz * (slice + 1) / nslices);
  const C2<R>* M = (const C2<R>*)P.inv + (long long)tile * P.bsz * P.bsz;
  for (int r = threadIdx.x; r < P.bsz; r += blockDim.x) {
    const long long d = tile_dof(P, tile, r);
    if (Q32) {
      const float2 v = P.q32[d];
      qs[r] = C2<R>{(R)v.x, (R)v.y};
    } else {
      const double2 v = P.q[d];
      qs[r] = C2<R>{(R)v.x, (R)v.y};
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool vec = sizeof(R) == 4 && (P.bsz & 1) == 0;
  for (int r = rb0 + wid; r < rb1; r += nw) {
    const C2<R>* row = M + (long long)r * P.bsz;
    R ar = 0, ai = 0;
    if (vec) {
      const float4* row4 = (const float4*)row;
      for (int c2 = lane; c2 < P.bsz / 2; c2 += 32) {
        const float4 m = __ldg(row4 + c2);
        const C2<R> x0 = qs[2 * c2], x1 = qs[2 * c2 + 1];
        ar += m.x * x0.x - m.y * x0.y + m.z * x1.x - m.w * x1.y;
        ai += m.x * x0.y + m.y * x0.x + m.z * x1.y + m.w * x1.x;
      }
    } else {
      for (int c = lane; c < P.bsz; c += 32) {
        C2<R> m = row[c], x = qs[c];
        ar += m.x * x.x - m.y * x.y;
        ai += m.x * x.y + m.y * x.x;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) P.z[tile_dof(P, tile, r)] = make_double2((double)ar, (double)ai);
  }
}

template <class R, bool Q32>
__global__ void k_apply_rows(const ApplyParams P) {
  if (P.gate && *P.gate) return;
  apply_rows_body<R, Q32>(P, blockIdx.x, blockIdx.y, gridDim.y);
}

// FP32 row-major blocks -> BF16 column-major blocks
__global__ void k_to_bf16_t(const float2* in, __nv_bfloat162* out, int b) {
  const float2* M = in + (long long)blockIdx.x * b * b;
  __nv_bfloat162* O = out + (long long)blockIdx.x * b * b;
  for (long long idx = threadIdx.x; idx < (long long)b * b; idx += blockDim.x) {
    const int c = (int)(idx / b), r = (int)(idx - (long long)c * b);  // write O[c][r] (coalesced)
    O[idx] = __float22bfloat162_rn(M[(long long)r * b + c]);
  }
}

// Batched apply over several handles (stab_jv_batch_precond_apply): item i
// owns the flat blocks [start[i], start[i+1]) = its (tile, row slice) grid
// with the tile fastest; V selects the storage layout (0 FP64 rows, 1 FP32
// rows, 2 BF16 four rows per thread, 3 BF16 one row per thread).
struct ApplyItem {
  ApplyParams P;
  long long ntiles;
};
static_assert(sizeof(ApplyItem) % 8 == 0, "items are copied to shared memory in 8-byte words");

template <int V>
__global__ void k_apply_batch(const ApplyItem* __restrict__ items, const int* __restrict__ start, int count) {
  __shared__ ApplyItem sI;
  int lo = 0, hi = count - 1;  // largest i with start[i] <= blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)__ldg(start + mid) <= blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const unsigned long long* src = (const unsigned long long*)(items + lo);
  for (int k = threadIdx.x; k < (int)(sizeof(ApplyItem) / 8); k += blockDim.x) ((unsigned long long*)&sI)[k] = __ldg(src + k);
  __syncthreads();
  if (sI.P.gate && *sI.P.gate) return;
  const long long local = (long long)blockIdx.x - __ldg(start + lo);
  const long long nt = sI.ntiles;
  const unsigned nslices = (unsigned)((__ldg(start + lo + 1) - __ldg(start + lo)) / nt);
  const long long tile = local % nt;
  const unsigned slice = (unsigned)(local / nt);
  if (V == 0) apply_rows_body<double, false>(sI.P, tile, slice, nslices);
  else if (V == 1) apply_rows_body<float, false>(sI.P, tile, slice, nslices);
  else if (V == 2) apply_cols4_body<false>(sI.P, tile, slice, nslices);
  else apply_cols_body<__nv_bfloat162, float, false>(sI.P, tile, slice, nslices);
}

struct Geo {
  int tx, ty, tz, ntx, nty, ntz, ntpts, bsz;
  long long ntiles;
};

// Tiles of the reduced-operator preconditioner (precond = 2): any tile that
// divides the grid with an even number of y points, levels of m = nv * 2 * tx * tz
// unknowns with m <= kBtMaxLevel.
constexpr int kBtMaxLevel = 256;
struct BtGeo {
  int m, nlev;
};
bool bt_geo(StabHandle* h, const Geo& g, BtGeo& b) {
  b.m = h->nv * 2 * g.tx * g.tz;
  b.nlev = g.ty / 2;
  return g.ty % 2 == 0 && b.m <= kBtMaxLevel;
}

bool tile_geo(StabHandle* h, Geo& g) {
  g.tx = h->opts.tile[0];
  g.ty = h->opts.tile[1];
  g.tz = h->dim == 3 ? h->opts.tile[2] : 1;
  if (g.tx < 1 || g.ty < 1 || g.tz < 1 || h->nx % g.tx || h->ny % g.ty || h->nz % g.tz) return false;
  g.ntx = h->nx / g.tx;
  g.nty = h->ny / g.ty;
  g.ntz = h->nz / g.tz;
  g.ntpts = g.tx * g.ty * g.tz;
  g.bsz = h->nv * g.ntpts;
  g.ntiles = (long long)g.ntx * g.nty * g.ntz;
  if (h->opts.precond == 2) {
    BtGeo b;
    return bt_geo(h, g, b);
  }
  return g.bsz <= 1024;
}

// The reduced operator's second-order explicit 1-D derivative matrices (same
// layout as the compact ones: [l * n + t] = (D e_l)_t) and its base table.
cudaError_t ensure_reduced(StabHandle* h) {
  cudaError_t e;
  for (int a = 0; a < h->dim; ++a) {
    if (h->d_dmat_low[a]) continue;
    const int n = h->ax[a].n;
    const double hh = h->ax[a].h;
    const bool per = h->ax[a].periodic;
    std::vector<double2> M((size_t)2 * n * n, make_double2(0.0, 0.0));
    auto put = [&](int which, int t, int l, double v) {
      if (per) l = (l % n + n) % n;
      M[(size_t)which * n * n + (size_t)l * n + t].x += v;
    };
    for (int t = 0; t < n; ++t) {
      if (per || (t > 0 && t < n - 1)) {
        put(0, t, t + 1, 1.0 / (2.0 * hh));
        put(0, t, t - 1, -1.0 / (2.0 * hh));
        put(1, t, t + 1, 1.0 / (hh * hh));
        put(1, t, t, -2.0 / (hh * hh));
        put(1, t, t - 1, 1.0 / (hh * hh));
      } else {
        const int sg = t == 0 ? 1 : -1;
        put(0, t, t, -3.0 * sg / (2.0 * hh));
        put(0, t, t + sg, 4.0 * sg / (2.0 * hh));
        put(0, t, t + 2 * sg, -1.0 * sg / (2.0 * hh));
        put(1, t, t, 2.0 / (hh * hh));
        put(1, t, t + sg, -5.0 / (hh * hh));
        put(1, t, t + 2 * sg, 4.0 / (hh * hh));
        put(1, t, t + 3 * sg, -1.0 / (hh * hh));
      }
    }
    double2* buf;
    if ((e = dalloc(h, &buf, M.size() * sizeof(double2))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(buf, M.data(), M.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
      dfree(h, buf);
      return e;
    }
    h->d_dmat_low[a] = (double*)buf;
  }
  if (!h->d_btab_low) {
    double* t;
    if ((e = dalloc(h, &t, (size_t)pw::bt_count(h->dim) * h->nbase * sizeof(double))) != cudaSuccess) return e;
    if ((e = jv_reduced_base_table(h, t)) != cudaSuccess) {
      dfree(h, t);
      return e;
    }
    h->d_btab_low = t;
  }
  return cudaSuccess;
}

cudaError_t ensure_dmats(StabHandle* h) {
  cudaError_t e;
  for (int a = 0; a < h->dim; ++a) {
    if (h->d_dmat[a]) continue;
    const int n = h->ax[a].n;
    double2* buf;
    if ((e = dalloc(h, &buf, (size_t)3 * n * n * sizeof(double2))) != cudaSuccess) return e;
    // [D1 | D2 | work]
    if ((e = jv_derivative_matrices(h, a, buf + (size_t)2 * n * n, buf, buf + (size_t)n * n)) != cudaSuccess) {
      dfree(h, buf);
      return e;
    }
    h->d_dmat[a] = (double*)buf;
  }
  return cudaSuccess;
}

AsmParams asm_params(StabHandle* h, const Geo& g, double2 sigma) {
  AsmParams P{};
  P.nx = h->nx; P.ny = h->ny; P.nz = h->nz;
  P.tx = g.tx; P.ty = g.ty; P.tz = g.tz; P.ntx = g.ntx; P.nty = g.nty; P.ntpts = g.ntpts; P.bsz = g.bsz;
  P.npts = h->npts; P.nbase = h->nbase; P.homog = h->homog;
  P.btab = h->d_btab;
  P.eta_y = h->d_metric;
  P.eta_yy = h->d_metric + h->ny;
  P.bcflags = h->d_bcflags;
  const bool red = h->opts.precond == 2;  // the reduced operator's tables
  if (red) P.btab = h->d_btab_low;
  for (int a = 0; a < 3; ++a) {
    P.nax[a] = h->ax[a].n;
    const int n = h->ax[a].n;
    const double* dm = red ? h->d_dmat_low[a] : h->d_dmat[a];
    P.Dm1[a] = a < h->dim ? (const double2*)dm : nullptr;
    P.Dm2[a] = a < h->dim ? (const double2*)dm + (size_t)n * n : nullptr;
  }
  if (h->dim == 2) { P.Dm1[2] = P.Dm1[0]; P.Dm2[2] = P.Dm2[0]; P.nax[2] = 1; }
  P.phys = phys_of(h);
  P.sigma = sigma;
  return P;
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion with partial pivoting whose trailing updates
// are batched complex GEMMs on the tensor cores (cuBLAS), FP32 blocks.
// Panel K = [k0, k0 + w): the w elimination steps on the panel columns only
// (pivot rows searched in all rows >= k, the in-place trick storing the
// transform's columns), which leaves the columns W = E_K[:, K] of the panel's
// block transform E_K = I + (W - I_K) e_K^T; the row interchanges are then
// applied to the other columns C and every other column is updated at once:
// A[:, C] <- E_K A[:, C] = A[:, C] + (W - I_K) A[K, C], i.e. with R = A[K, C]
// saved and A[K, C] set to zero, A[:, C] += W R (one GEMM per side of K).
// Two levels: the panels of an outer block of PB columns update only the
// columns of that outer block (GEMMs with K = one panel); the outer block's
// transform, accumulated in its PB columns in the same in-place form, then
// updates every other column (GEMMs with K = PB).  Both levels are the same
// identity applied to nested column sets, so the result is the unblocked
// sweep's up to rounding.  The column interchanges are undone at the end.
// ---------------------------------------------------------------------------
constexpr int kPanelThreads = 256;

// The panel's w steps on a copy of the b x w panel in shared memory (one CTA
// per block; row stride w + 1 complex so that column sweeps spread over the
// banks), written back at the end.  piv[k] receives the pivot row of step k.
template <int W>
__global__ void __launch_bounds__(kPanelThreads) k_gj_panel(float2* A, int b, int k0, int w, int* piv, int* info) {
  extern __shared__ float2 Ps[];  // [b][W + 1]
  __shared__ double rv[kPanelThreads / 32];
  __shared__ int ri[kPanelThreads / 32];
  __shared__ int s_piv;
  __shared__ float2 s_row[W];
  __shared__ float2 s_inv;
  constexpr int LD = W + 1;
  float2* M = A + (long long)blockIdx.x * b * b;
  int* pv = piv + (long long)blockIdx.x * b;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int idx = threadIdx.x; idx < b * w; idx += blockDim.x) {
    const int i = idx / w, c = idx - i * w;
    Ps[i * LD + c] = M[(long long)i * b + k0 + c];
  }
  __syncthreads();
  int bad = 0;
  for (int kk = 0; kk < w; ++kk) {
    const int k = k0 + kk;
    double best = -1.0;
    int bi = b;
    for (int i = k + threadIdx.x; i < b; i += blockDim.x) {
      const float2 v = Ps[i * LD + kk];
      const double m = (double)v.x * v.x + (double)v.y * v.y;
      if (m > best) { best = m; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = -1.0;
      int bbi = b;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q)
        if (rv[q] > bb || (rv[q] == bb && ri[q] < bbi)) { bb = rv[q]; bbi = ri[q]; }
      if (!(bb > 0.0)) { bad = k + 1; bbi = k; }
      s_piv = bbi;
      pv[k] = bbi;
    }
    __syncthreads();
    const int p = s_piv;
    // swap rows k and p of the panel; row k (after the interchange) to s_row
    if (threadIdx.x < w) {
      const float2 a = Ps[k * LD + threadIdx.x], d = Ps[p * LD + threadIdx.x];
      if (p != k) Ps[p * LD + threadIdx.x] = a;
      s_row[threadIdx.x] = d;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const float2 q = s_row[kk];
      float den = q.x * q.x + q.y * q.y;
      if (!(den > 0.0f)) den = 1.0f;
      s_inv = make_float2(q.x / den, -q.y / den);
    }
    __syncthreads();
    const float2 inv = s_inv;
    if (threadIdx.x < w) {  // row k: divided by the pivot, the pivot position becomes 1 / pivot
      const float2 q = threadIdx.x == kk ? make_float2(1.0f, 0.0f) : s_row[threadIdx.x];
      const float2 r = make_float2(q.x * inv.x - q.y * inv.y, q.x * inv.y + q.y * inv.x);
      s_row[threadIdx.x] = r;
      Ps[k * LD + threadIdx.x] = r;
    }
    __syncthreads();
    // the other rows: a_ic -= a_ik r_c, a_ik taken as zero in the pivot column (in-place trick); the
    // thread of (i, kk) owns the multiplier a_ik, so every row's threads read it before it changes
    for (int idx = threadIdx.x; idx < b * w; idx += blockDim.x) {
      const int i = idx / w, c = idx - i * w;
      if (i == k || c == kk) continue;
      const float2 f = Ps[i * LD + kk];
      const float2 r = s_row[c];
      float2& a = Ps[i * LD + c];
      a = make_float2(a.x - (f.x * r.x - f.y * r.y), a.y - (f.x * r.y + f.y * r.x));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
      if (i == k) continue;
      const float2 f = Ps[i * LD + kk];
      const float2 r = s_row[kk];
      Ps[i * LD + kk] = make_float2(-(f.x * r.x - f.y * r.y), -(f.x * r.y + f.y * r.x));
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < b * w; idx += blockDim.x) {
    const int i = idx / w, c = idx - i * w;
    M[(long long)i * b + k0 + c] = Ps[i * LD + c];
  }
  if (threadIdx.x == 0 && bad) atomicMax(info, 1);
}

// The row interchanges of steps [r0, r0 + rw) on the columns C = [lo, hi)
// outside K = [r0, r0 + rw), then T[kk][j] = A[r0 + kk][j] for j in C (saved,
// row length b) and A[K, C] = 0.  Thread j owns column j.
__global__ void k_gj_swap_copy(float2* A, int b, int r0, int rw, int lo, int hi, const int* piv, float2* T,
                               long long tstride) {
  float2* M = A + (long long)blockIdx.x * b * b;
  const int* pv = piv + (long long)blockIdx.x * b;
  float2* Tb = T + (long long)blockIdx.x * tstride;
  for (int j = lo + threadIdx.x; j < hi; j += blockDim.x) {
    if (j >= r0 && j < r0 + rw) continue;
    for (int kk = 0; kk < rw; ++kk) {
      const int k = r0 + kk, p = pv[k];
      if (p != k) {
        const float2 a = M[(long long)k * b + j];
        M[(long long)k * b + j] = M[(long long)p * b + j];
        M[(long long)p * b + j] = a;
      }
    }
    for (int kk = 0; kk < rw; ++kk) {
      Tb[(long long)kk * b + j] = M[(long long)(r0 + kk) * b + j];
      M[(long long)(r0 + kk) * b + j] = make_float2(0.0f, 0.0f);
    }
  }
}

// Undo the row interchanges: swap columns in reverse order (thread i owns row i).
__global__ void k_gj_unpermute(float2* A, int b, const int* piv) {
  float2* M = A + (long long)blockIdx.x * b * b;
  const int* pv = piv + (long long)blockIdx.x * b;
  for (int i = threadIdx.x; i < b; i += blockDim.x)
    for (int k = b - 1; k >= 0; --k) {
      const int p = pv[k];
      if (p != k) {
        const float2 t = M[(long long)i * b + k];
        M[(long long)i * b + k] = M[(long long)i * b + p];
        M[(long long)i * b + p] = t;
      }
    }
}

int gj_threads(int b) {
  int t = b < 512 ? b : 512;
  return ((t + 31) / 32) * 32;  // whole warps: the pivot search reduces with full-warp shuffles
}

cudaError_t launch_assemble(StabHandle* h, AsmParams& P, long long ntile_batch) {
  if (h->dim == 2) k_assemble<2><<<(unsigned)ntile_batch, 128, 0, h->stream>>>(P);
  else k_assemble<3><<<(unsigned)ntile_batch, 128, 0, h->stream>>>(P);
  return cudaGetLastError();
}

// Outer block width of the two-level sweep (a multiple of both panel widths).
int gj_outer(int b) { return b <= 512 ? 128 : 256; }

// In-place inversion of nb FP32 blocks (b x b, row-major) by the blocked
// Gauss-Jordan sweep above; mode 1: GEMMs with FP32 inputs emulated on the
// BF16 tensor cores (BF16x9, FP32 accuracy), mode 2: TF32 tensor cores.
// T holds gj_outer(b) x b complex values per block.
cudaError_t gj_blocked(StabHandle* h, float2* A, int b, long long nb, int* piv, float2* T, int* d_info, int mode) {
  if (!h->cublas) {
    cublasHandle_t c;
    if (cublasCreate(&c) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    h->cublas = c;
  }
  cublasHandle_t cb = (cublasHandle_t)h->cublas;
  if (cublasSetStream(cb, h->stream) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
  cublasComputeType_t ct = CUBLAS_COMPUTE_32F_FAST_TF32;
  if (mode == 1) {
    ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    cublasSetEmulationStrategy(cb, CUBLAS_EMULATION_STRATEGY_EAGER);
  }
  // panels of 32 columns while the b x 33 panel fits in shared memory (b <= 640), else 16
  const int W = b <= 640 ? 32 : 16;
  const int PB = gj_outer(b);
  const long long tstride = (long long)PB * b;
  const size_t psm = (size_t)b * (W + 1) * sizeof(float2);
  cudaError_t ea = cudaFuncSetAttribute(W == 32 ? (const void*)k_gj_panel<32> : (const void*)k_gj_panel<16>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
  if (ea != cudaSuccess) return ea;
  const cuComplex one = make_cuComplex(1.0f, 0.0f);
  // rows [r0, r0 + rw) eliminated: interchanges, T and zeroing on [lo, hi) outside them, then
  // (column-major view X = A^T, ld b) X[C, :] += T^T[C, :] X[K, :] for C left and right of K
  auto update = [&](int r0, int rw, int lo, int hi) -> cudaError_t {
    k_gj_swap_copy<<<(unsigned)nb, 256, 0, h->stream>>>(A, b, r0, rw, lo, hi, piv, T, tstride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int side = 0; side < 2; ++side) {
      const int c0 = side == 0 ? lo : r0 + rw;
      const int m = side == 0 ? r0 - lo : hi - (r0 + rw);
      if (m <= 0) continue;
      const cublasStatus_t st = cublasGemmStridedBatchedEx(
          cb, CUBLAS_OP_N, CUBLAS_OP_N, m, b, rw, &one, T + c0, CUDA_C_32F, b, tstride, A + r0, CUDA_C_32F, b,
          (long long)b * b, &one, A + c0, CUDA_C_32F, b, (long long)b * b, (int)nb, ct, CUBLAS_GEMM_DEFAULT);
      if (st != CUBLAS_STATUS_SUCCESS) return st == CUBLAS_STATUS_NOT_SUPPORTED ? cudaErrorNotSupported : cudaErrorUnknown;
    }
    return cudaSuccess;
  };
  for (int o0 = 0; o0 < b; o0 += PB) {
    const int ow = std::min(PB, b - o0);
    for (int k0 = o0; k0 < o0 + ow; k0 += W) {
      const int w = std::min(W, o0 + ow - k0);
      if (W == 32) k_gj_panel<32><<<(unsigned)nb, kPanelThreads, psm, h->stream>>>(A, b, k0, w, piv, d_info);
      else k_gj_panel<16><<<(unsigned)nb, kPanelThreads, psm, h->stream>>>(A, b, k0, w, piv, d_info);
      cudaError_t e = update(k0, w, o0, o0 + ow);
      if (e != cudaSuccess) return e;
    }
    if (ow < b) {
      cudaError_t e = update(o0, ow, 0, b);
      if (e != cudaSuccess) return e;
    }
  }
  k_gj_unpermute<<<(unsigned)nb, 256, 0, h->stream>>>(A, b, piv);
  return cudaGetLastError();
}

}  // namespace

cudaError_t pc_block(StabHandle* h, double2 sigma, long long t, double2* d_out) {
  Geo g;
  if (!tile_geo(h, g) || t < 0 || t >= g.ntiles) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = h->opts.precond == 2 ? ensure_reduced(h) : ensure_dmats(h)) != cudaSuccess) return e;
  AsmParams P = asm_params(h, g, sigma);
  P.tile0 = t;
  P.out = d_out;
  return launch_assemble(h, P, 1);
}

// Reduced-operator preconditioner: the tiles' level blocks assembled in FP64
// in batches of at most ~1 GiB, factorised by block Thomas elimination in the
// storage precision (FP32 or FP64).
cudaError_t pc_build_reduced(StabHandle* h, const Geo& g, double2 sigma) {
  BtGeo bg;
  if (!bt_geo(h, g, bg)) return cudaErrorInvalidValue;
  cudaError_t e;
  if ((e = ensure_reduced(h)) != cudaSuccess) return e;
  const int prec = h->opts.precond_prec == 64 ? 64 : 32;
  const size_t esz = prec == 64 ? sizeof(double2) : sizeof(float2);
  const size_t per = (size_t)bg.nlev * 3 * bg.m * bg.m;  // complex values per tile
  if (!h->d_pinv || h->ntiles != g.ntiles || h->bsize != -(long long)bg.m * bg.nlev || h->pprec != prec) {
    dfree(h, h->d_pinv);
    h->d_pinv = nullptr;
    if ((e = dalloc(h, &h->d_pinv, per * g.ntiles * esz)) != cudaSuccess) return e;
    h->ntiles = g.ntiles;
    h->bsize = -(long long)bg.m * bg.nlev;  // negative: block-tridiagonal layout
    h->pprec = prec;
  }
  h->pvalid = false;
  long long batch = (long long)((1ull << 30) / (per * sizeof(double2)));
  if (batch < 1) batch = 1;
  if (batch > g.ntiles) batch = g.ntiles;
  double2* asmb;
  if ((e = dalloc(h, &asmb, per * batch * sizeof(double2))) != cudaSuccess) return e;
  int* d_info;
  if ((e = dalloc(h, &d_info, sizeof(int))) != cudaSuccess) { dfree(h, asmb); return e; }
  cudaMemsetAsync(d_info, 0, sizeof(int), h->stream);
  AsmParams P = asm_params(h, g, sigma);
  const size_t smem = (size_t)2 * bg.m * esz + (size_t)bg.m * sizeof(int);
  for (long long t0 = 0; t0 < g.ntiles && e == cudaSuccess; t0 += batch) {
    const long long nb = std::min(batch, g.ntiles - t0);
    P.tile0 = t0;
    const dim3 grid((unsigned)nb, (unsigned)bg.nlev, 3u);
    if (h->dim == 2) k_assemble_bt<2><<<grid, 128, 0, h->stream>>>(P, bg.m, bg.nlev, asmb);
    else k_assemble_bt<3><<<grid, 128, 0, h->stream>>>(P, bg.m, bg.nlev, asmb);
    if (prec == 64)
      k_bt_factor<double><<<(unsigned)nb, 256, smem, h->stream>>>(asmb, (C2<double>*)h->d_pinv + per * t0, bg.m,
                                                                    bg.nlev, d_info);
    else
      k_bt_factor<float><<<(unsigned)nb, 256, smem, h->stream>>>(asmb, (C2<float>*)h->d_pinv + per * t0, bg.m,
                                                                   bg.nlev, d_info);
    e = cudaGetLastError();
  }
  int info = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, d_info);
  dfree(h, asmb);
  if (e != cudaSuccess) return e;
  if (info) return cudaErrorInvalidValue;
  h->psigma_re = sigma.x;
  h->psigma_im = sigma.y;
  h->pvalid = true;
  return cudaSuccess;
}

cudaError_t pc_build(StabHandle* h, double2 sigma) {
  Geo g;
  if (!tile_geo(h, g)) return cudaErrorInvalidValue;
  if (h->opts.precond == 2) return pc_build_reduced(h, g, sigma);
  cudaError_t e;
  if ((e = ensure_dmats(h)) != cudaSuccess) return e;
  const int prec = h->opts.precond_prec;
  const size_t esz = prec == 64 ? sizeof(double2) : prec == 32 ? sizeof(float2) : sizeof(__nv_bfloat162);
  const size_t bb = (size_t)g.bsz * g.bsz;
  if (!h->d_pinv || h->ntiles != g.ntiles || h->bsize != g.bsz || h->pprec != prec) {
    dfree(h, h->d_pinv);
    h->d_pinv = nullptr;
    if ((e = dalloc(h, &h->d_pinv, bb * g.ntiles * esz)) != cudaSuccess) return e;
    h->ntiles = g.ntiles;
    h->bsize = g.bsz;
    h->pprec = prec;
  }
  h->pvalid = false;
  // FP64 assembly in batches of at most ~1 GiB (directly into the inverse storage when FP64)
  long long batch = (long long)((1ull << 30) / (bb * sizeof(double2)));
  if (batch < 1) batch = 1;
  if (batch > g.ntiles) batch = g.ntiles;
  if (prec != 64 && !h->d_pblk) {
    if ((e = dalloc(h, &h->d_pblk, bb * batch * sizeof(double2))) != cudaSuccess) return e;
  }
  float2* f32 = nullptr;  // BF16 storage: FP32 inversion in a batch-sized buffer, then rounding
  if (prec == 16 && (e = dalloc(h, &f32, bb * batch * sizeof(float2))) != cudaSuccess) return e;
  const int fac = h->opts.precond_factor;  // 1, 2: blocked sweep with tensor-core GEMMs (FP32 inversion only)
  int* piv = nullptr;
  float2* T = nullptr;
  if (fac && prec != 64) {
    if ((e = dalloc(h, &piv, (size_t)batch * g.bsz * sizeof(int))) != cudaSuccess) return e;
    if ((e = dalloc(h, &T, (size_t)batch * gj_outer(g.bsz) * g.bsz * sizeof(float2))) != cudaSuccess) return e;
  }
  int* d_info;
  if ((e = dalloc(h, &d_info, sizeof(int))) != cudaSuccess) return e;
  cudaMemsetAsync(d_info, 0, sizeof(int), h->stream);
  AsmParams P = asm_params(h, g, sigma);
  const size_t smem = (size_t)2 * g.bsz * (prec == 64 ? sizeof(double2) : sizeof(float2)) + g.bsz * sizeof(int);
  for (long long t0 = 0; t0 < g.ntiles; t0 += batch) {
    const long long nb = std::min(batch, g.ntiles - t0);
    P.tile0 = t0;
    if (prec == 64) {
      P.out = (double2*)h->d_pinv + bb * t0;
      if ((e = launch_assemble(h, P, nb)) != cudaSuccess) break;
      k_gauss_jordan<double><<<(unsigned)nb, gj_threads(g.bsz), smem, h->stream>>>(
          (C2<double>*)P.out, g.bsz, d_info);
    } else {
      P.out = h->d_pblk;
      if ((e = launch_assemble(h, P, nb)) != cudaSuccess) break;
      float2* dst = prec == 32 ? (float2*)h->d_pinv + bb * t0 : f32;
      k_to_float<<<1024, 256, 0, h->stream>>>(h->d_pblk, dst, (long long)(bb * nb));
      if (fac) {
        if ((e = gj_blocked(h, dst, g.bsz, nb, piv, T, d_info, fac)) != cudaSuccess) break;
      } else {
        k_gauss_jordan<float><<<(unsigned)nb, gj_threads(g.bsz), smem, h->stream>>>((C2<float>*)dst, g.bsz, d_info);
      }
      if (prec == 16)
        k_to_bf16_t<<<(unsigned)nb, 256, 0, h->stream>>>(f32, (__nv_bfloat162*)h->d_pinv + bb * t0, g.bsz);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) break;
  }
  int info = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, d_info);
  dfree(h, f32);
  dfree(h, piv);
  dfree(h, T);
  if (e != cudaSuccess) return e;
  if (info) return cudaErrorInvalidValue;  // a singular block
  h->pvalid = true;
  h->psigma_re = sigma.x;
  h->psigma_im = sigma.y;
  h->stats.precond_builds++;
  return cudaSuccess;
}

cudaError_t pc_apply(StabHandle* h, const double2* q, double2* z, const float2* q32) {
  if (!h->pvalid) return cudaErrorInvalidValue;
  Geo g;
  tile_geo(h, g);
  if (h->opts.precond == 2) {
    BtGeo bg;
    bt_geo(h, g, bg);
    BtApplyParams B{};
    B.q = q; B.q32 = q32; B.z = z; B.F = h->d_pinv;
    B.m = bg.m; B.nlev = bg.nlev; B.tx = g.tx; B.ty = g.ty; B.tz = g.tz; B.ntx = g.ntx; B.nty = g.nty;
    B.nx = h->nx; B.ny = h->ny; B.npts = h->npts; B.gate = h->gate;
    const int ts = phase_begin(h, STAB_PHASE_PRECOND_APPLY);
    const dim3 grid_rhs((unsigned)g.ntiles, (unsigned)bg.nlev);
    const unsigned nt = (unsigned)g.ntiles;
    // threads per row of the 256-thread products, and the row fragment length
    int G = 1;
    while (G < 32 && 2 * G * bg.m <= 256) G *= 2;
    const int frag = (bg.m + G - 1) / G;
    if (h->pprec == 64) {
      const size_t sm = 2 * bg.m * sizeof(double2);
      if (frag <= 8) {
        if (q32) k_bt_rhs<double, true, 8><<<grid_rhs, 256, sm, h->stream>>>(B);
        else k_bt_rhs<double, false, 8><<<grid_rhs, 256, sm, h->stream>>>(B);
        k_bt_sweep<double, 8><<<nt, 256, sm, h->stream>>>(B);
      } else {
        if (q32) k_bt_rhs<double, true, 0><<<grid_rhs, 256, sm, h->stream>>>(B);
        else k_bt_rhs<double, false, 0><<<grid_rhs, 256, sm, h->stream>>>(B);
        k_bt_sweep<double, 0><<<nt, 256, sm, h->stream>>>(B);
      }
    } else {
      const size_t sm = 2 * bg.m * sizeof(float2);
      if (frag <= 16) {
        if (q32) k_bt_rhs<float, true, 16><<<grid_rhs, 256, sm, h->stream>>>(B);
        else k_bt_rhs<float, false, 16><<<grid_rhs, 256, sm, h->stream>>>(B);
        k_bt_sweep<float, 16><<<nt, 256, sm, h->stream>>>(B);
      } else {
        if (q32) k_bt_rhs<float, true, 0><<<grid_rhs, 256, sm, h->stream>>>(B);
        else k_bt_rhs<float, false, 0><<<grid_rhs, 256, sm, h->stream>>>(B);
        k_bt_sweep<float, 0><<<nt, 256, sm, h->stream>>>(B);
      }
    }
    phase_end(h, ts);
    return cudaGetLastError();
  }
  ApplyParams P{};
  P.q = q; P.z = z; P.inv = h->d_pinv; P.q32 = q32;
  P.nx = h->nx; P.ny = h->ny; P.tx = g.tx; P.ty = g.ty; P.tz = g.tz; P.ntx = g.ntx; P.nty = g.nty;
  P.ntpts = g.ntpts; P.bsz = g.bsz; P.npts = h->npts;
  P.gate = h->gate;
  const int ts = phase_begin(h, STAB_PHASE_PRECOND_APPLY);
  // row slices so that small grids still spread over the SMs.  FP64 / FP32 storage is
  // row-major (a warp per row), BF16 column-major (a thread per row): measured fastest each
  int slices = (int)((2 * 152 + g.ntiles - 1) / g.ntiles);
  slices = std::max(1, std::min(slices, g.bsz / 32));
  const dim3 grid((unsigned)g.ntiles, (unsigned)slices);
  // the input's precision is a template parameter (FP32 basis: float2 input)
  const bool q32v = q32 != nullptr;
  if (h->pprec == 64) {
    if (q32v) k_apply_rows<double, true><<<grid, 256, g.bsz * sizeof(double2), h->stream>>>(P);
    else k_apply_rows<double, false><<<grid, 256, g.bsz * sizeof(double2), h->stream>>>(P);
  } else if (h->pprec == 32) {
    if (q32v) k_apply_rows<float, true><<<grid, 256, g.bsz * sizeof(float2), h->stream>>>(P);
    else k_apply_rows<float, false><<<grid, 256, g.bsz * sizeof(float2), h->stream>>>(P);
  } else if (g.bsz % 4 == 0) {
    const int quads = (g.bsz / 4 + slices - 1) / slices;
    const int thr = std::min(256, ((quads + 31) / 32) * 32);
    if (q32v) k_apply_cols4<true><<<grid, thr, g.bsz * sizeof(float2), h->stream>>>(P);
    else k_apply_cols4<false><<<grid, thr, g.bsz * sizeof(float2), h->stream>>>(P);
  } else {
    const int rows = (g.bsz + slices - 1) / slices;
    const int thr = std::min(256, ((rows + 31) / 32) * 32);
    if (q32v) k_apply_cols<__nv_bfloat162, float, true><<<grid, thr, g.bsz * sizeof(float2), h->stream>>>(P);
    else k_apply_cols<__nv_bfloat162, float, false><<<grid, thr, g.bsz * sizeof(float2), h->stream>>>(P);
  }
  phase_end(h, ts);
  return cudaGetLastError();
}

extern "C" stab_status stab_precond_build(stab_handle hh, double sr, double si) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  Geo g;
  if (!tile_geo(h, g)) { h->err = h->opts.precond == 2 ? "stab_precond_build: tile must divide the grid, with an even ty and levels of at most 256 unknowns (nv * 2 * tx * tz)" : "stab_precond_build: tile must divide the grid and give blocks of at most 1024 unknowns"; return STAB_ERR_INVALID_ARG; }
  cudaError_t e = pc_build(h, make_double2(sr, si));
  if (e == cudaErrorInvalidValue) { h->err = "stab_precond_build: singular block"; return STAB_ERR_NUMERIC; }
  if (e != cudaSuccess) { h->err = std::string("stab_precond_build: ") + cudaGetErrorString(e); return e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA; }
  return STAB_OK;
}

extern "C" stab_status stab_precond_apply(stab_handle hh, const void* q, void* z) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  if (!q || !z || q == z) { h->err = "stab_precond_apply: bad vectors"; return STAB_ERR_INVALID_ARG; }
  if (!h->pvalid) { h->err = "stab_precond_apply: preconditioner not built"; return STAB_ERR_INVALID_ARG; }
  cudaError_t e = pc_apply(h, (const double2*)q, (double2*)z);
  if (e != cudaSuccess) { h->err = std::string("stab_precond_apply: ") + cudaGetErrorString(e); return STAB_ERR_CUDA; }
  return STAB_OK;
}

extern "C" stab_status stab_precond_block(stab_handle hh, double sr, double si, long long t, double* out) {
  StabHandle* h = (StabHandle*)hh;
  if (!h) return STAB_ERR_INVALID_ARG;
  Geo g;
  if (!out || !tile_geo(h, g) || t < 0 || t >= g.ntiles) { h->err = "stab_precond_block: bad tile or output"; return STAB_ERR_INVALID_ARG; }
  double2* d;
  cudaError_t e = dalloc(h, &d, (size_t)g.bsz * g.bsz * sizeof(double2));
  if (e == cudaSuccess) e = pc_block(h, make_double2(sr, si), t, d);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)g.bsz * g.bsz * sizeof(double2), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, d);
  if (e != cudaSuccess) { h->err = std::string("stab_precond_block: ") + cudaGetErrorString(e); return STAB_ERR_CUDA; }
  return STAB_OK;
}

// Batched block apply: one launch per storage layout for all instances.
cudaError_t pc_batch_plan(const std::vector<StabHandle*>& hs, const double2* const* q, double2* const* z,
                          const int* const* gates, BatchImage& im, PcBatchPlan& plan) {
  const int count = (int)hs.size();
  std::vector<ApplyItem> items[4];
  std::vector<int> blocks[4];
  int threads[4] = {0, 0, 0, 0};
  size_t smem[4] = {0, 0, 0, 0};
  for (int i = 0; i < count; ++i) {
    StabHandle* h = hs[i];
    if (!h->pvalid) return cudaErrorInvalidValue;
    if (h->opts.precond == 2) return cudaErrorNotSupported;  // block-tridiagonal tiles: single-handle apply only
    Geo g;
    tile_geo(h, g);
    ApplyItem it{};
    ApplyParams& P = it.P;
    P.q = q[i]; P.z = z[i]; P.inv = h->d_pinv; P.q32 = nullptr;
    P.nx = h->nx; P.ny = h->ny; P.tx = g.tx; P.ty = g.ty; P.tz = g.tz; P.ntx = g.ntx; P.nty = g.nty;
    P.ntpts = g.ntpts; P.bsz = g.bsz; P.npts = h->npts;
    P.gate = gates ? gates[i] : nullptr;
    it.ntiles = g.ntiles;
    // the same slices and threads as the single-handle apply
    int slices = (int)((2 * 152 + g.ntiles - 1) / g.ntiles);
    slices = std::max(1, std::min(slices, g.bsz / 32));
    int var, thr;
    size_t sm;
    if (h->pprec == 64) { var = 0; thr = 256; sm = g.bsz * sizeof(double2); }
    else if (h->pprec == 32) { var = 1; thr = 256; sm = g.bsz * sizeof(float2); }
    else if (g.bsz % 4 == 0) {
      var = 2;
      const int quads = (g.bsz / 4 + slices - 1) / slices;
      thr = std::min(256, ((quads + 31) / 32) * 32);
      sm = g.bsz * sizeof(float2);
    } else {
      var = 3;
      const int rows = (g.bsz + slices - 1) / slices;
      thr = std::min(256, ((rows + 31) / 32) * 32);
      sm = g.bsz * sizeof(float2);
    }
    if (g.ntiles * slices > (1LL << 30)) return cudaErrorInvalidValue;
    items[var].push_back(it);
    blocks[var].push_back((int)(g.ntiles * slices));
    threads[var] = std::max(threads[var], thr);
    smem[var] = std::max(smem[var], sm);
  }
  for (int v = 0; v < 4; ++v) plan.sec[v] = im.section(items[v], blocks[v], threads[v], smem[v]);
  return im.overflow ? cudaErrorInvalidValue : cudaSuccess;
}

cudaError_t pc_batch_launch(const PcBatchPlan& plan, const unsigned char* d, cudaStream_t st) {
  for (int v = 0; v < 4; ++v) {
    const BatchSection& S = plan.sec[v];
    if (!S.count) continue;
    const ApplyItem* it = (const ApplyItem*)(d + S.items);
    const int* sp = (const int*)(d + S.start);
    if (v == 0) k_apply_batch<0><<<S.blocks, S.threads, S.smem, st>>>(it, sp, S.count);
    else if (v == 1) k_apply_batch<1><<<S.blocks, S.threads, S.smem, st>>>(it, sp, S.count);
    else if (v == 2) k_apply_batch<2><<<S.blocks, S.threads, S.smem, st>>>(it, sp, S.count);
    else k_apply_batch<3><<<S.blocks, S.threads, S.smem, st>>>(it, sp, S.count);
  }
  return cudaGetLastError();
}

cudaError_t pc_apply_batch(stab_jv_batch_s* B, const double2* const* q, double2* const* z) {
  BatchImage im;
  PcBatchPlan plan;
  cudaError_t e = pc_batch_plan(B->hs, q, z, nullptr, im, plan);
  if (e != cudaSuccess) return e;
  if ((e = batch_stage(B, im)) != cudaSuccess) return e;
  if ((e = batch_order_begin(B)) != cudaSuccess) return e;
  if ((e = pc_batch_launch(plan, (const unsigned char*)B->d_buf, B->stream)) != cudaSuccess) return e;
  return batch_order_end(B);
}

extern "C" stab_status stab_jv_batch_precond_apply(stab_jv_batch B, const void* const* q, void* const* z) {
  if (!B) return STAB_ERR_INVALID_ARG;
  if (!q || !z) {
    B->err = "stab_jv_batch_precond_apply: null vector list";
    return STAB_ERR_INVALID_ARG;
  }
  const int count = (int)B->hs.size();
  for (int i = 0; i < count; ++i) {
    const char* a = (const char*)q[i];
    const char* b = (const char*)z[i];
    const long long bytes = B->hs[i]->n * (long long)sizeof(double2);
    if (!a || !b || (a < b + bytes && b < a + bytes)) {
      B->err = "stab_jv_batch_precond_apply: null or overlapping q / z of instance " + std::to_string(i);
      return STAB_ERR_INVALID_ARG;
    }
    if (!B->hs[i]->pvalid) {
      B->err = "stab_jv_batch_precond_apply: no preconditioner built for instance " + std::to_string(i);
      return STAB_ERR_INVALID_ARG;
    }
    if (B->hs[i]->opts.precond == 2) {
      B->err = "stab_jv_batch_precond_apply: instance " + std::to_string(i) + " uses the reduced-operator preconditioner";
      return STAB_ERR_UNSUPPORTED;
    }
  }
  const cudaError_t e = pc_apply_batch(B, (const double2* const*)q, (double2* const*)z);
  if (e != cudaSuccess) {
    B->err = std::string("stab_jv_batch_precond_apply: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STAB_ERR_OOM : STAB_ERR_CUDA;
  }
  return STAB_OK;
}
