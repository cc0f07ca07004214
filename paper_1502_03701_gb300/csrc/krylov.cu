// Krylov kernels: batched complex dot products (V^H w) with a fixed-order
// two-stage reduction, V h updates, CGS2 (classical Gram-Schmidt twice), the
// tall-skinny basis product V Q of the implicit restart, and vector helpers.
// Vectors are complex128 (double2); a basis V of k vectors stores column j at
// V + j*n.
#include "internal.cuh"
#include "pairs.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// partial[b * k + j] = sum over this block's rows of conj(V_j[i]) w[i]
__global__ void __launch_bounds__(kThreads) k_dot_partial(const double2* __restrict__ V, int k, long long n,
                                                         const double2* __restrict__ w, double2* partial) {
  __shared__ double red[2][kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < k; ++j) {
    const double2* Vj = V + (long long)j * n;
    double sr = 0.0, si = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      double2 a = Vj[i], b = w[i];
      sr = fma(a.x, b.x, fma(a.y, b.y, sr));   // Re(conj(a) b)
      si = fma(a.x, b.y, fma(-a.y, b.x, si));  // Im(conj(a) b)
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) { red[0][wid] = sr; red[1][wid] = si; }
    __syncthreads();
    if (wid == 0) {
      double tr = lane < kThreads / 32 ? red[0][lane] : 0.0;
      double ti = lane < kThreads / 32 ? red[1][lane] : 0.0;
      tr = warp_sum(tr);
      ti = warp_sum(ti);
      if (lane == 0) partial[(long long)blockIdx.x * k + j] = make_double2(tr, ti);
    }
    __syncthreads();
  }
}

// out[j] (+)= sum_b partial[b * k + j], fixed order; one warp per column
__global__ void k_dot_final(const double2* partial, int nb, int k, double2* out, int accumulate) {
  const int j = blockIdx.x;
  double sr = 0.0, si = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) {
    double2 p = partial[(long long)b * k + j];
    sr += p.x;
    si += p.y;
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if (threadIdx.x == 0) {
    if (accumulate) { out[j].x += sr; out[j].y += si; }
    else out[j] = make_double2(sr, si);
  }
}

// w[i] -= sum_j V_j[i] h[j]   (sign = -1)   or   x[i] += sum_j V_j[i] y[j]   (sign = +1)
// (kdev, when set, lowers k to *kdev: the column count is known only on the device)
__global__ void __launch_bounds__(kThreads) k_gemv(const double2* __restrict__ V, int k, long long n,
                                                  const double2* __restrict__ h, double2* x, double sign,
                                                  const int* kdev) {
  if (kdev) k = min(k, *kdev);
  extern __shared__ double2 hs[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double ar = 0.0, ai = 0.0;
    for (int j = 0; j < k; ++j) {
      double2 a = V[(long long)j * n + i], c = hs[j];
      ar = fma(a.x, c.x, fma(-a.y, c.y, ar));
      ai = fma(a.x, c.y, fma(a.y, c.x, ai));
    }
    double2 xv = x[i];
    x[i] = make_double2(fma(sign, ar, xv.x), fma(sign, ai, xv.y));
  }
}

// x = x / *d_norm  (into out if given); gate as in the J v kernels
__global__ void k_scale_inv(double2* x, long long n, const double* d_norm, double2* out, const int* gate) {
  if (gate && *gate) return;
  const double s = 1.0 / *d_norm;
  double2* o = out ? out : x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 v = x[i];
    o[i] = make_double2(v.x * s, v.y * s);
  }
}

// y = a x + b y (complex a, b)
__global__ void k_axpby(double2 a, const double2* x, double2 b, double2* y, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 xv = x[i], yv = y[i];
    y[i] = make_double2(a.x * xv.x - a.y * xv.y + b.x * yv.x - b.y * yv.y,
                        a.x * xv.y + a.y * xv.x + b.x * yv.y + b.y * yv.x);
  }
}

// tmp_j[i] = sum_l V_l[i] Q[l + j*m] for j < kk (Q column-major m x kk).  A
// block stages its rows of V (rows x m) in shared memory once.
constexpr int kVqRows = 64;
__global__ void __launch_bounds__(kVqRows) k_vq(const double2* __restrict__ V, int m, long long n,
                                               const double2* __restrict__ Q, int kk, double2* tmp) {
  extern __shared__ double2 vs[];  // [m][kVqRows]
  const long long i0 = (long long)blockIdx.x * kVqRows;
  const long long i = i0 + threadIdx.x;
  for (int l = 0; l < m; ++l) vs[l * kVqRows + threadIdx.x] = i < n ? V[(long long)l * n + i] : make_double2(0.0, 0.0);
  __syncthreads();
  if (i >= n) return;
  for (int j = 0; j < kk; ++j) {
    double ar = 0.0, ai = 0.0;
    for (int l = 0; l < m; ++l) {
      double2 a = vs[l * kVqRows + threadIdx.x], q = __ldg(&Q[(long long)j * m + l]);
      ar = fma(a.x, q.x, fma(-a.y, q.y, ar));
      ai = fma(a.x, q.y, fma(a.y, q.x, ai));
    }
    tmp[(long long)j * n + i] = make_double2(ar, ai);
  }
}

// ---------------------------------------------------------------------------
// Fused CGS2.  Block b owns the contiguous rows [r0, r1) of every vector.
// Pass A: partial1 = per-block sums of V^H w.  Pass B: every block reduces
// partial1 to h1 (same fixed order in every block), updates its rows
// w -= V h1 and forms its sums of V^H w' (partial2).  Pass C: every block
// reduces partial2 to h2, updates w -= V h2 and forms its sum of |w|^2;
// block 0 stores h = h1 + h2.  A final warp sums the norm partials.
// Dot products: one warp per column (a warp group per column when k is
// smaller than the warp count), so no block barrier is taken per column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_partials(const double2* partial, int nb, int k, double2* hs) {
  // hs[j] = sum_b partial[b * k + j]; one warp per column, fixed order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < k; j += nw) {
    double sr = 0.0, si = 0.0;
    for (int b = lane; b < nb; b += 32) {
      double2 p = partial[(long long)b * k + j];
      sr += p.x;
      si += p.y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) hs[j] = make_double2(sr, si);
  }
}

// Columns with j % kFp64Every == kFp64Every - 1 are formed with native FP64
// FMAs, the others in pair arithmetic: the pair path keeps the integer and
// FP32 pipes busy, the FP64 pipe (1/58 of FP32 on GB300) takes the rest.
constexpr int kFp64Every = 4;
__device__ __forceinline__ bool fp64_column(int j) { return j % kFp64Every == kFp64Every - 1; }

// sum over rows [q0, q1) of conj(x_i) w_i by one warp: exact FP32
// two-products of the integer-split pairs, accumulated by two-sum (or FP64
// FMAs for the FP64 columns); every lane returns the warp's total.
__device__ __forceinline__ double2 warp_dot(const double2* __restrict__ x, const double2* __restrict__ w, long long q0,
                                            long long q1, bool fp64) {
  const int lane = threadIdx.x & 31;
  if (fp64) {
    double sr = 0.0, si = 0.0;
#pragma unroll 4
    for (long long i = q0 + lane; i < q1; i += 32) {
      const double2 a = x[i], b = w[i];
      sr = fma(a.x, b.x, fma(a.y, b.y, sr));
      si = fma(a.x, b.y, fma(-a.y, b.x, si));
    }
    return make_double2(warp_sum(sr), warp_sum(si));
  }
  ffn sr{0.0f, 0.0f}, si{0.0f, 0.0f};
#pragma unroll 4
  for (long long i = q0 + lane; i < q1; i += 32) {
    const double2 av = x[i], bv = w[i];
    const ffn ar = ff_split(av.x), ai = ff_split(av.y), br = ff_split(bv.x), bi = ff_split(bv.y);
    ff_acc_prod(sr, ar, br);             // Re conj(a) b = ar br + ai bi
    ff_acc_prod(sr, ai, bi);
    ff_acc_prod(si, ar, bi);             // Im conj(a) b = ar bi - ai br
    ff_acc_prod(si, ff_negate(ai), br);
  }
  sr = ff_warp_sum(sr);
  si = ff_warp_sum(si);
  return make_double2(ff_to_d(sr), ff_to_d(si));
}

// partial_out[b * k + j] = this block's sum of conj(V_j) w over [r0, r1).
// red: shared, one double2 per warp.  Block-uniform control flow.
// FP32 basis: FP32 FMAs per lane, FP64 across lanes (the basis itself carries FP32 precision)
__device__ __forceinline__ double2 warp_dot32(const float2* __restrict__ x, const float2* __restrict__ w, long long q0,
                                              long long q1) {
  const int lane = threadIdx.x & 31;
  float sr = 0.f, si = 0.f;
#pragma unroll 4
  for (long long i = q0 + lane; i < q1; i += 32) {
    const float2 a = x[i], b = w[i];
    sr = fmaf(a.x, b.x, fmaf(a.y, b.y, sr));
    si = fmaf(a.x, b.y, fmaf(-a.y, b.x, si));
  }
  return make_double2(warp_sum((double)sr), warp_sum((double)si));
}

__device__ __forceinline__ double2 col_dot(const double2* x, const double2* w, long long q0, long long q1, int j) {
  return warp_dot(x, w, q0, q1, fp64_column(j));
}
__device__ __forceinline__ double2 col_dot(const float2* x, const float2* w, long long q0, long long q1, int) {
  return warp_dot32(x, w, q0, q1);
}

template <class T>
__device__ __forceinline__ void block_dot_columns(const T* __restrict__ V, int k, long long n, long long r0,
                                                  long long r1, const T* w, double2* partial_out, double2* red,
                                                  unsigned bidx) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (k >= nw) {
    for (int j = wid; j < k; j += nw) {
      const double2 d = col_dot(V + (long long)j * n, w, r0, r1, j);
      if (lane == 0) partial_out[(long long)bidx * k + j] = d;
    }
    return;
  }
  const int G = nw / k;  // warps per column, each over a fixed sub-range
  double2 d = make_double2(0.0, 0.0);
  if (wid < G * k) {
    const int j = wid / G, sg = wid - j * G;
    const long long len = r1 - r0;
    d = col_dot(V + (long long)j * n, w, r0 + len * sg / G, r0 + len * (sg + 1) / G, j);
  }
  if (lane == 0) red[wid] = d;
  __syncthreads();
  if ((int)threadIdx.x < k) {
    const int j = threadIdx.x;
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < G; ++q) {
      sr += red[j * G + q].x;
      si += red[j * G + q].y;
    }
    partial_out[(long long)bidx * k + j] = make_double2(sr, si);
  }
  __syncthreads();
}

// w_i -= sum_j V_j[i] h_j for one row: pair arithmetic with h as pairs in
// shared memory, FP64 FMAs for the FP64 columns (h in FP64 in shared memory).
__device__ __forceinline__ double2 row_update(const double2* __restrict__ V, int k, long long n, long long i,
                                              const double2* h64, const ffn* hre, const ffn* him, double2 wv) {
  ffn ar{0.0f, 0.0f}, ai{0.0f, 0.0f};
  double dr = 0.0, di = 0.0;
#pragma unroll 4
  for (int j = 0; j < k; ++j) {
    const double2 a = V[(long long)j * n + i];
    if (fp64_column(j)) {
      const double2 c = h64[j];
      dr = fma(a.x, c.x, fma(-a.y, c.y, dr));
      di = fma(a.x, c.y, fma(a.y, c.x, di));
      continue;
    }
    const ffn xr = ff_split(a.x), xi = ff_split(a.y);
    ff_acc_prod(ar, xr, hre[j]);            // Re(a h) = ar hr - ai hi
    ff_acc_prod(ar, ff_negate(xi), him[j]);
    ff_acc_prod(ai, xr, him[j]);            // Im(a h) = ar hi + ai hr
    ff_acc_prod(ai, xi, hre[j]);
  }
  return make_double2(wv.x - (ff_to_d(ar) + dr), wv.y - (ff_to_d(ai) + di));
}

// rows [r0, r1) of block bidx of nb (equal contiguous ranges)
__device__ __forceinline__ void block_rows(long long n, long long& r0, long long& r1, unsigned bidx, unsigned nb) {
  const long long rows = (n + nb - 1) / nb;
  r0 = (long long)bidx * rows;
  r1 = r0 + rows < n ? r0 + rows : n;
}

// The three CGS2 steps and the final norm for block bidx of nb (one
// instance's launch, or one item of a batched launch).
__device__ __forceinline__ void cgs2_a_body(const double2* __restrict__ V, int k, long long n,
                                            const double2* __restrict__ w, double2* partial1, unsigned bidx,
                                            unsigned nb) {
  __shared__ double2 red[kThreads / 32];
  long long r0, r1;
  block_rows(n, r0, r1, bidx, nb);
  block_dot_columns(V, k, n, r0, r1, w, partial1, red, bidx);
}

__device__ __forceinline__ void cgs2_b_body(const double2* __restrict__ V, int k, long long n, double2* w,
                                            const double2* partial1, double2* partial2, double2* d_h, unsigned bidx,
                                            unsigned nb) {
  extern __shared__ double2 hs[];  // k complex, then 2k pairs
  __shared__ double2 red[kThreads / 32];
  ffn* hre = (ffn*)(hs + k);
  ffn* him = hre + k;
  reduce_partials(partial1, nb, k, hs);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    hre[j] = ff_split(hs[j].x);
    him[j] = ff_split(hs[j].y);
    if (bidx == 0) d_h[j] = hs[j];
  }
  __syncthreads();
  long long r0, r1;
  block_rows(n, r0, r1, bidx, nb);
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) w[i] = row_update(V, k, n, i, hs, hre, him, w[i]);
  __syncthreads();  // this block's rows of w are final; the dots below read only them
  block_dot_columns(V, k, n, r0, r1, w, partial2, red, bidx);
}

__device__ __forceinline__ void cgs2_c_body(const double2* __restrict__ V, int k, long long n, double2* w,
                                            const double2* partial2, double2* d_h, double* norm_partial,
                                            unsigned bidx, unsigned nb) {
  extern __shared__ double2 hs[];  // k complex, then 2k pairs
  __shared__ double red[kThreads / 32];
  ffn* hre = (ffn*)(hs + k);
  ffn* him = hre + k;
  reduce_partials(partial2, nb, k, hs);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    hre[j] = ff_split(hs[j].x);
    him[j] = ff_split(hs[j].y);
    if (bidx == 0) {
      double2 h1 = d_h[j];
      d_h[j] = make_double2(h1.x + hs[j].x, h1.y + hs[j].y);
    }
  }
  __syncthreads();
  long long r0, r1;
  block_rows(n, r0, r1, bidx, nb);
  double s = 0.0;
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double2 r = row_update(V, k, n, i, hs, hre, him, w[i]);
    w[i] = r;
    s = fma(r.x, r.x, fma(r.y, r.y, s));
  }
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (wid == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) norm_partial[bidx] = t;
  }
}

__device__ __forceinline__ void norm_final_body(const double* partial, int nb, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += partial[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void __launch_bounds__(kThreads) k_cgs2_a(const double2* __restrict__ V, int k, long long n,
                                                    const double2* __restrict__ w, double2* partial1,
                                                    const int* gate) {
  if (gate && *gate) return;
  cgs2_a_body(V, k, n, w, partial1, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads) k_cgs2_b(const double2* __restrict__ V, int k, long long n, double2* w,
                                                    const double2* partial1, double2* partial2, double2* d_h,
                                                    const int* gate) {
  if (gate && *gate) return;
  cgs2_b_body(V, k, n, w, partial1, partial2, d_h, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kThreads) k_cgs2_c(const double2* __restrict__ V, int k, long long n, double2* w,
                                                    const double2* partial2, double2* d_h, double* norm_partial,
                                                    const int* gate) {
  if (gate && *gate) return;
  cgs2_c_body(V, k, n, w, partial2, d_h, norm_partial, blockIdx.x, gridDim.x);
}

__global__ void k_norm_final(const double* partial, int nb, double* out, const int* gate) {
  if (gate && *gate) return;
  norm_final_body(partial, nb, out);
}

// Batched CGS2 over several handles (stab_jv_batch_orthogonalize): item i
// owns the flat blocks [start[i], start[i+1]) (its own block count nb, so its
// row ranges and reduction order are those of its single launch).
struct CgsItem {
  const double2* V;
  double2* w;
  double2* p1;
  double2* p2;
  double2* d_h;
  double* np;
  double* d_norm;
  const int* gate;  // per-instance gate of a batched solver (nullable)
  long long n;
  int k, nb;
};
static_assert(sizeof(CgsItem) % 8 == 0, "items are read as 8-byte words");

__device__ __forceinline__ int cgs_item(const int* __restrict__ start, int count, unsigned b) {
  int lo = 0, hi = count - 1;  // largest i with start[i] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kThreads) k_cgs2_a_batch(const CgsItem* __restrict__ items,
                                                          const int* __restrict__ start, int count) {
  const int i = cgs_item(start, count, blockIdx.x);
  const CgsItem it = items[i];
  if (it.gate && *it.gate) return;
  cgs2_a_body(it.V, it.k, it.n, it.w, it.p1, blockIdx.x - (unsigned)__ldg(start + i), (unsigned)it.nb);
}

__global__ void __launch_bounds__(kThreads) k_cgs2_b_batch(const CgsItem* __restrict__ items,
                                                          const int* __restrict__ start, int count) {
  const int i = cgs_item(start, count, blockIdx.x);
  const CgsItem it = items[i];
  if (it.gate && *it.gate) return;
  cgs2_b_body(it.V, it.k, it.n, it.w, it.p1, it.p2, it.d_h, blockIdx.x - (unsigned)__ldg(start + i),
              (unsigned)it.nb);
}

__global__ void __launch_bounds__(kThreads) k_cgs2_c_batch(const CgsItem* __restrict__ items,
                                                          const int* __restrict__ start, int count) {
  const int i = cgs_item(start, count, blockIdx.x);
  const CgsItem it = items[i];
  if (it.gate && *it.gate) return;
  cgs2_c_body(it.V, it.k, it.n, it.w, it.p2, it.d_h, it.np, blockIdx.x - (unsigned)__ldg(start + i),
              (unsigned)it.nb);
}

// one 32-thread block per item
__global__ void k_norm_final_batch(const CgsItem* __restrict__ items, int count) {
  if ((int)blockIdx.x >= count) return;
  const CgsItem it = items[blockIdx.x];
  if (it.gate && *it.gate) return;
  norm_final_body(it.np, it.nb, it.d_norm);
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt with selective reorthogonalisation (Daniel, Gragg,
// Kaufman and Stewart 1976) for the GMRES basis: one pass h1 = V^H w,
// w' = w - V h1; a second pass only when ||w'|| < eta ||w|| (eta = 1/sqrt 2),
// decided on the device; the second-pass kernels return at once otherwise.
// Same dot and update arithmetic as the fused CGS2 kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool gated(const int* a, const int* b) { return (a && *a) || (b && *b); }

__device__ __forceinline__ double norm2_of(double2 z) { return z.x * z.x + z.y * z.y; }
__device__ __forceinline__ double norm2_of(float2 z) { return (double)fmaf(z.x, z.x, z.y * z.y); }

template <class T>
__device__ __forceinline__ double block_norm_partial(const T* w, long long r0, long long r1, double* red) {
  double s = 0.0;
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) s += norm2_of(w[i]);
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  double t = 0.0;
  if (wid == 0) {
    t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// pass-1 dots and the block's |w|^2
template <class T>
__global__ void __launch_bounds__(kThreads) k_dgks_dots(const T* __restrict__ V, int k, long long n,
                                                       const T* __restrict__ w, double2* partial,
                                                       double* norm_partial, const int* gate, const int* skip) {
  if (gated(gate, skip)) return;
  __shared__ double2 red[kThreads / 32];
  __shared__ double rn[kThreads / 32];
  long long r0, r1;
  block_rows(n, r0, r1, blockIdx.x, gridDim.x);
  block_dot_columns(V, k, n, r0, r1, w, partial, red, blockIdx.x);
  if (norm_partial) {
    const double t = block_norm_partial(w, r0, r1, rn);
    if (threadIdx.x == 0) norm_partial[blockIdx.x] = t;
  }
}

// h = reduced partial dots (block 0 stores or adds it to d_h), w -= V h over
// the block's rows, the block's |w|^2
__global__ void __launch_bounds__(kThreads) k_dgks_update(const double2* __restrict__ V, int k, long long n,
                                                         double2* w, const double2* partial, double2* d_h,
                                                         double* norm_partial, int accumulate, const int* gate,
                                                         const int* skip) {
  if (gated(gate, skip)) return;
  extern __shared__ double2 hs[];  // k complex, then 2k pairs
  __shared__ double red[kThreads / 32];
  ffn* hre = (ffn*)(hs + k);
  ffn* him = hre + k;
  reduce_partials(partial, gridDim.x, k, hs);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    hre[j] = ff_split(hs[j].x);
    him[j] = ff_split(hs[j].y);
    if (blockIdx.x == 0) {
      if (accumulate) {
        const double2 h1 = d_h[j];
        d_h[j] = make_double2(h1.x + hs[j].x, h1.y + hs[j].y);
      } else {
        d_h[j] = hs[j];
      }
    }
  }
  __syncthreads();
  long long r0, r1;
  block_rows(n, r0, r1, blockIdx.x, gridDim.x);
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) w[i] = row_update(V, k, n, i, hs, hre, him, w[i]);
  __syncthreads();
  const double t = block_norm_partial(w, r0, r1, red);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = t;
}

// ||w||, ||w'|| from the partials; skip = (||w'|| >= eta ||w||); when skipping,
// ||w'|| is the result
__global__ void k_dgks_decide(const double* np0, const double* np1, int nb, double* d_norm, int* skip, double eta,
                              const int* gate) {
  if (gate && *gate) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) {
    a += np0[i];
    b += np1[i];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (threadIdx.x == 0) {
    const double n0 = sqrt(a), n1 = sqrt(b);
    const int s = n1 >= eta * n0;  // NaN: reorthogonalise (and let the norm report it)
    *skip = s;
    if (s) *d_norm = n1;
  }
}

__global__ void k_dgks_norm(const double* partial, int nb, double* out, const int* gate, const int* skip) {
  if (gated(gate, skip)) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) s += partial[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *out = sqrt(s);
}

// FP32 basis: h = reduced partials (block 0 stores or adds it to d_h in
// FP64), w -= V h in FP32 over the block's rows, the block's |w|^2.
__global__ void __launch_bounds__(kThreads) k_dgks32_update(const float2* __restrict__ V, int k, long long n, float2* w,
                                                           const double2* partial, double2* d_h, double* norm_partial,
                                                           int accumulate, const int* gate, const int* skip) {
  if (gated(gate, skip)) return;
  extern __shared__ double2 hs[];  // k complex (FP64), then k float2
  __shared__ double red[kThreads / 32];
  float2* hf = (float2*)(hs + k);
  reduce_partials(partial, gridDim.x, k, hs);
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    hf[j] = make_float2((float)hs[j].x, (float)hs[j].y);
    if (blockIdx.x == 0) {
      if (accumulate) {
        const double2 h1 = d_h[j];
        d_h[j] = make_double2(h1.x + hs[j].x, h1.y + hs[j].y);
      } else {
        d_h[j] = hs[j];
      }
    }
  }
  __syncthreads();
  long long r0, r1;
  block_rows(n, r0, r1, blockIdx.x, gridDim.x);
  for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    float ar = 0.f, ai = 0.f;
#pragma unroll 4
    for (int j = 0; j < k; ++j) {
      const float2 a = V[(long long)j * n + i], c = hf[j];
      ar = fmaf(a.x, c.x, fmaf(-a.y, c.y, ar));
      ai = fmaf(a.x, c.y, fmaf(a.y, c.x, ai));
    }
    const float2 wv = w[i];
    w[i] = make_float2(wv.x - ar, wv.y - ai);
  }
  __syncthreads();
  const double t = block_norm_partial(w, r0, r1, red);
  if (threadIdx.x == 0) norm_partial[blockIdx.x] = t;
}

// out (FP32) = in (FP64) / *d_norm (d_norm may be NULL: plain rounding); gated
__global__ void k_to_f32(const double2* in, long long n, const double* d_norm, float2* out, const int* gate) {
  if (gate && *gate) return;
  const double s = d_norm ? 1.0 / *d_norm : 1.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = in[i];
    out[i] = make_float2((float)(v.x * s), (float)(v.y * s));
  }
}

// out (FP64) = in (FP32); gated
__global__ void k_to_f64(const float2* in, long long n, double2* out, const int* gate) {
  if (gate && *gate) return;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i].x, in[i].y);
}

// x (FP32) /= *d_norm in place; gated
__global__ void k_scale32(float2* x, long long n, const double* d_norm, const int* gate) {
  if (gate && *gate) return;
  const float s = (float)(1.0 / *d_norm);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = x[i];
    x[i] = make_float2(v.x * s, v.y * s);
  }
}

// out (FP64) = sum_{j < min(k, *kdev)} V_j y_j over an FP32 basis (FP32 products)
__global__ void __launch_bounds__(kThreads) k_gemv32(const float2* __restrict__ V, int k, const int* kdev, long long n,
                                                    const double2* __restrict__ y, double2* out) {
  if (kdev) k = min(k, *kdev);
  extern __shared__ float2 ys[];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = make_float2((float)y[j].x, (float)y[j].y);
  __syncthreads();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float ar = 0.f, ai = 0.f;
#pragma unroll 4
    for (int j = 0; j < k; ++j) {
      const float2 a = V[(long long)j * n + i], c = ys[j];
      ar = fmaf(a.x, c.x, fmaf(-a.y, c.y, ar));
      ai = fmaf(a.x, c.y, fmaf(a.y, c.x, ai));
    }
    out[i] = make_double2(ar, ai);
  }
}

// blocks of the fused CGS2: about 64 rows each (short latency on small
// vectors), at most four per SM on large ones
int cgs_blocks(long long n) {
  long long b = (n + 63) / 64;
  if (b > 152 * 4) b = 152 * 4;
  return (int)(b < 1 ? 1 : b);
}

int red_blocks(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 4) b = 152 * 4;
  return (int)(b < 1 ? 1 : b);
}

int grid_n(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t kry_dot(StabHandle* h, const double2* V, int k, long long n, const double2* w, double2* d_h,
                            double2* partial, int accumulate) {
  const int nb = red_blocks(n);
  k_dot_partial<<<nb, kThreads, 0, h->stream>>>(V, k, n, w, partial);
  k_dot_final<<<k, 32, 0, h->stream>>>(partial, nb, k, d_h, accumulate);
  return cudaGetLastError();
}

cudaError_t kry_gemv_sub(StabHandle* h, const double2* V, int k, long long n, const double2* d_h, double2* w) {
  if (k <= 0) return cudaSuccess;
  k_gemv<<<grid_n(n), kThreads, k * sizeof(double2), h->stream>>>(V, k, n, d_h, w, -1.0, nullptr);
  return cudaGetLastError();
}

cudaError_t kry_gemv_add(StabHandle* h, const double2* V, int k, long long n, const double2* d_y, double2* x,
                         const int* kdev) {
  if (k <= 0) return cudaSuccess;
  k_gemv<<<grid_n(n), kThreads, k * sizeof(double2), h->stream>>>(V, k, n, d_y, x, 1.0, kdev);
  return cudaGetLastError();
}

// CGS2: h = V^H w; w -= V h; h2 = V^H w; w -= V h2; h += h2; *d_norm = ||w||.
// partial holds kry_partial_elems(n, k) complex (two sets of block sums and
// the norm partials); d_h holds 2k complex.
cudaError_t kry_cgs2(StabHandle* h, const double2* V, int k, long long n, double2* w, double2* d_h, double* d_norm,
                     double2* partial) {
  const int nb = cgs_blocks(n);
  double2* p1 = partial;
  double2* p2 = partial + (size_t)nb * (k > 0 ? k : 1);
  double* np = (double*)(p2 + (size_t)nb * (k > 0 ? k : 1));
  const int ts = phase_begin(h, STAB_PHASE_CGS2);
  cudaError_t e;
  if (k > 0) {
    const size_t sm = (size_t)k * (sizeof(double2) + 2 * sizeof(ffn));
    k_cgs2_a<<<nb, kThreads, 0, h->stream>>>(V, k, n, w, p1, h->gate);
    k_cgs2_b<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p1, p2, d_h, h->gate);
    k_cgs2_c<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p2, d_h, np, h->gate);
    k_norm_final<<<1, 32, 0, h->stream>>>(np, nb, d_norm, h->gate);
    e = cudaGetLastError();
  } else {
    e = launch_norm2(h, w, n, d_norm, 1);
  }
  phase_end(h, ts);
  return e;
}

cudaError_t kry_scale(StabHandle* h, double2* x, long long n, const double* d_norm, double2* out) {
  k_scale_inv<<<grid_n(n), kThreads, 0, h->stream>>>(x, n, d_norm, out, h->gate);
  return cudaGetLastError();
}

cudaError_t kry_axpby(StabHandle* h, double2 a, const double2* x, double2 b, double2* y, long long n) {
  k_axpby<<<grid_n(n), kThreads, 0, h->stream>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t kry_copy(StabHandle* h, const double2* x, double2* y, long long n) {
  return cudaMemcpyAsync(y, x, n * sizeof(double2), cudaMemcpyDeviceToDevice, h->stream);
}

// tmp[:, 0:kk] = V[:, 0:m] Q  (Q device, column-major m x kk)
cudaError_t kry_update_basis(StabHandle* h, double2* V, int m, int kk, long long n, const double2* d_Q, double2* tmp) {
  const size_t smem = (size_t)m * kVqRows * sizeof(double2);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  k_vq<<<(unsigned)((n + kVqRows - 1) / kVqRows), kVqRows, smem, h->stream>>>(V, m, n, d_Q, kk, tmp);
  return cudaGetLastError();
}

int kry_dgks_partial_elems(long long n, int k) {
  const int nb = cgs_blocks(n);
  return 2 * nb * (k > 0 ? k : 1) + (3 * nb + 1) / 2 + 2;
}

// GMRES orthogonalisation with selective reorthogonalisation (see the kernels):
// h (k complex in d_h) and ||w|| (d_norm); partial holds kry_dgks_partial_elems.
cudaError_t kry_dgks(StabHandle* h, const double2* V, int k, long long n, double2* w, double2* d_h, double* d_norm,
                     double2* partial) {
  if (k <= 0) return kry_cgs2(h, V, k, n, w, d_h, d_norm, partial);
  const int ts = phase_begin(h, STAB_PHASE_CGS2);
  const int nb = cgs_blocks(n);
  double2* p1 = partial;
  double2* p2 = partial + (size_t)nb * k;
  double* np0 = (double*)(p2 + (size_t)nb * k);
  double* np1 = np0 + nb;
  double* np2 = np1 + nb;
  int* skip = (int*)(np2 + nb);
  const size_t sm = (size_t)k * (sizeof(double2) + 2 * sizeof(ffn));
  constexpr double eta = 0.70710678118654752;
  k_dgks_dots<double2><<<nb, kThreads, 0, h->stream>>>(V, k, n, w, p1, np0, h->gate, nullptr);
  k_dgks_update<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p1, d_h, np1, 0, h->gate, nullptr);
  k_dgks_decide<<<1, 32, 0, h->stream>>>(np0, np1, nb, d_norm, skip, eta, h->gate);
  k_dgks_dots<double2><<<nb, kThreads, 0, h->stream>>>(V, k, n, w, p2, nullptr, h->gate, skip);
  k_dgks_update<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p2, d_h, np2, 1, h->gate, skip);
  k_dgks_norm<<<1, 32, 0, h->stream>>>(np2, nb, d_norm, h->gate, skip);
  phase_end(h, ts);
  return cudaGetLastError();
}

// FP32 basis: the selective Gram-Schmidt of kry_dgks in FP32 arithmetic
// (h and ||w|| in FP64); partial holds kry_dgks_partial_elems complex.
cudaError_t kry_dgks32(StabHandle* h, const float2* V, int k, long long n, float2* w, double2* d_h, double* d_norm,
                       double2* partial) {
  const int ts = phase_begin(h, STAB_PHASE_CGS2);
  const int nb = cgs_blocks(n);
  double2* p1 = partial;
  double2* p2 = partial + (size_t)nb * k;
  double* np0 = (double*)(p2 + (size_t)nb * k);
  double* np1 = np0 + nb;
  double* np2 = np1 + nb;
  int* skip = (int*)(np2 + nb);
  const size_t sm = (size_t)k * (sizeof(double2) + sizeof(float2));
  constexpr double eta = 0.70710678118654752;
  k_dgks_dots<float2><<<nb, kThreads, 0, h->stream>>>(V, k, n, w, p1, np0, h->gate, nullptr);
  k_dgks32_update<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p1, d_h, np1, 0, h->gate, nullptr);
  k_dgks_decide<<<1, 32, 0, h->stream>>>(np0, np1, nb, d_norm, skip, eta, h->gate);
  k_dgks_dots<float2><<<nb, kThreads, 0, h->stream>>>(V, k, n, w, p2, nullptr, h->gate, skip);
  k_dgks32_update<<<nb, kThreads, sm, h->stream>>>(V, k, n, w, p2, d_h, np2, 1, h->gate, skip);
  k_dgks_norm<<<1, 32, 0, h->stream>>>(np2, nb, d_norm, h->gate, skip);
  phase_end(h, ts);
  return cudaGetLastError();
}

cudaError_t kry_to_f32(StabHandle* h, const double2* in, long long n, const double* d_norm, float2* out) {
  k_to_f32<<<grid_n(n), kThreads, 0, h->stream>>>(in, n, d_norm, out, h->gate);
  return cudaGetLastError();
}

cudaError_t kry_to_f64(StabHandle* h, const float2* in, long long n, double2* out) {
  k_to_f64<<<grid_n(n), kThreads, 0, h->stream>>>(in, n, out, h->gate);
  return cudaGetLastError();
}

cudaError_t kry_scale32(StabHandle* h, float2* x, long long n, const double* d_norm) {
  k_scale32<<<grid_n(n), kThreads, 0, h->stream>>>(x, n, d_norm, h->gate);
  return cudaGetLastError();
}

cudaError_t kry_gemv32(StabHandle* h, const float2* V, int k, const int* kdev, long long n, const double2* y,
                       double2* out) {
  k_gemv32<<<grid_n(n), kThreads, k * sizeof(float2), h->stream>>>(V, k, kdev, n, y, out);
  return cudaGetLastError();
}

// kernel attributes of this file, set for the current device at handle creation
cudaError_t kry_init_attributes() {
  return cudaFuncSetAttribute(k_vq, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int kry_partial_elems(long long n, int k) {
  const int nb = cgs_blocks(n);
  return 2 * nb * (k > 0 ? k : 1) + (nb + 1) / 2 + 1;
}

// CGS2 on an explicit stream with caller-provided scratch (no handle):
// partial needs red_blocks(n) * k complex, d_h 2k complex, norm_partial
// ceil(n / 1024) (at most 1024) doubles.  The same classical Gram-Schmidt
// applied twice as kry_cgs2, computed with the separate dot / update kernels.
cudaError_t kry_cgs2_stream(cudaStream_t st, const double2* V, int k, long long n, double2* w, double2* d_h,
                            double* d_norm, double2* partial, double* norm_partial, int norm_blocks) {
  if (k > 0) {
    const int nb = red_blocks(n);
    for (int pass = 0; pass < 2; ++pass) {
      double2* hp = d_h + (size_t)pass * k;
      k_dot_partial<<<nb, kThreads, 0, st>>>(V, k, n, w, partial);
      k_dot_final<<<k, 32, 0, st>>>(partial, nb, k, hp, 0);
      k_gemv<<<grid_n(n), kThreads, k * sizeof(double2), st>>>(V, k, n, hp, w, -1.0, nullptr);
    }
    k_axpby<<<1, 64, 0, st>>>(make_double2(1.0, 0.0), d_h + k, make_double2(1.0, 0.0), d_h, k);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_norm2_stream(st, w, n, norm_partial, norm_blocks, d_norm);
}

// Parameter image of a batched CGS2 (job i gated by J.gate) and its launches.
cudaError_t cgs2_batch_plan(const std::vector<CgsJob>& jobs, BatchImage& im, CgsBatchPlan& plan) {
  std::vector<CgsItem> items;
  std::vector<int> blocks, ones;
  size_t sm = 0;
  for (const CgsJob& J : jobs) {
    if (J.k < 1) return cudaErrorInvalidValue;
    const int nb = cgs_blocks(J.n);
    CgsItem it{};
    it.V = J.V;
    it.w = J.w;
    it.p1 = J.partial;
    it.p2 = J.partial + (size_t)nb * J.k;
    it.np = (double*)(it.p2 + (size_t)nb * J.k);
    it.d_h = J.d_h;
    it.d_norm = J.d_norm;
    it.gate = J.gate;
    it.n = J.n;
    it.k = J.k;
    it.nb = nb;
    items.push_back(it);
    blocks.push_back(nb);
    ones.push_back(1);
    sm = std::max(sm, (size_t)J.k * (sizeof(double2) + 2 * sizeof(ffn)));
  }
  plan.S = im.section(items, blocks, kThreads, sm);
  plan.N = im.section(items, ones, 32, 0);
  plan.sm = sm;
  return im.overflow ? cudaErrorInvalidValue : cudaSuccess;
}

cudaError_t cgs2_batch_launch(const CgsBatchPlan& plan, const unsigned char* d, cudaStream_t st) {
  if (!plan.S.count) return cudaSuccess;
  const CgsItem* it = (const CgsItem*)(d + plan.S.items);
  const int* sp = (const int*)(d + plan.S.start);
  k_cgs2_a_batch<<<plan.S.blocks, kThreads, 0, st>>>(it, sp, plan.S.count);
  k_cgs2_b_batch<<<plan.S.blocks, kThreads, plan.sm, st>>>(it, sp, plan.S.count);
  k_cgs2_c_batch<<<plan.S.blocks, kThreads, plan.sm, st>>>(it, sp, plan.S.count);
  k_norm_final_batch<<<plan.N.count, 32, 0, st>>>((const CgsItem*)(d + plan.N.items), plan.N.count);
  return cudaGetLastError();
}

// Batched CGS2: w_i <- (I - V_i V_i^H)^2 w_i for every job, one launch per
// step for all of them on the batch's stream.  Job i uses the same scratch
// layout and block count as kry_cgs2 (k >= 1), so its results are those of
// the single call.
cudaError_t kry_cgs2_batch(stab_jv_batch_s* B, const std::vector<CgsJob>& jobs) {
  BatchImage im;
  CgsBatchPlan plan;
  cudaError_t e = cgs2_batch_plan(jobs, im, plan);
  if (e != cudaSuccess) return e;
  if ((e = batch_stage(B, im)) != cudaSuccess) return e;
  if ((e = batch_order_begin(B)) != cudaSuccess) return e;
  if ((e = cgs2_batch_launch(plan, (const unsigned char*)B->d_buf, B->stream)) != cudaSuccess) return e;
  return batch_order_end(B);
}
