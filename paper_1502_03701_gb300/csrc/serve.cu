// Many stability problems on one GPU (no counterpart in the paper, which
// solves one problem at a time):
//  * stab_eigs_batch: the Cayley-IRAM solves of several handles run side by
//    side, one host thread and one private stream per handle, each solve's
//    GMRES cycles replayed from its own captured CUDA graph;
//  * stab_server_*: continuous batching of solve requests of any grid size
//    and flow parameters: a request is admitted when a slot is free and its
//    estimated device memory fits the budget; admitted requests' kernels
//    overlap on the device; a slot takes the next request as soon as its
//    solve ends.
// Every solve uses exactly the kernels and reduction orders of a lone
// stab_eigs call on the same handle configuration, so its results do not
// depend on what else runs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "pointwise.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// slot count of the J v scratch (see make_slots in jv.cu)
long long scratch_fields(int D, bool visc) {
  long long c = 1;  // temperature perturbation
  for (int ax = 0; ax < D; ++ax) c += (visc ? D + 3 : D + 2) + (visc ? D + 1 : 0);
  if (visc) c += (long long)D * (D - 1);
  return c;
}

}  // namespace

extern "C" long long stab_estimate_bytes(const stab_grid* g, const stab_opts* opts, int yonly, int nev, int ncv) {
  if (!g || g->dim < 2 || g->dim > 3 || g->nx < 1 || g->ny < 1 || g->nz < 1) return -1;
  stab_opts o;
  if (opts) o = *opts;
  else stab_default_opts(&o);
  const int D = g->dim;
  const long long npts = (long long)g->nx * g->ny * g->nz, nv = D + 2, n = nv * npts;
  const bool visc = true;  // the estimate covers the viscous (larger) case
  const long long nbase = yonly ? g->ny : npts;
  long long b = 0;
  b += n * 8;                                              // q0
  b += (long long)pw::bt_count(D) * nbase * (8 + 4);       // base tables, FP64 and FP32
  b += scratch_fields(D, visc) * npts * 16;                // derivative fields
  b += (nv + 1) * npts * 16;                               // set-up temporary
  const long long m = o.gmres_m, pc = o.precond != 0;
  if (o.gmres_basis_prec == 32) b += (m + 1) * n * 8 + 6 * n * 16;  // FP32 basis; r, b, x, w, z, t
  else if (o.gmres_inner_m > 0)                            // nested: V, Z, r, b, x; inner FP32 basis, w, zt, t
    b += ((m + 1) + m + 3) * n * 16 + ((long long)o.gmres_inner_m + 1) * n * 8 + 3 * n * 16;
  else if (o.lgmres_k > 0) b += ((m + 1) + m + 3 + 2 * (long long)o.lgmres_k + 1) * n * 16;  // LGMRES: V, Z, r, b,
                                                                                       // x, (z, A z) pairs, dz
  else b += ((m + 1) + pc * m + 3) * n * 16;               // GMRES basis, Z, r, b, x
  b += 2 * 608 * (m + 2) * 16;                             // CGS2 partial sums
  b += ((long long)ncv + 2 + nev + 1) * n * 16;            // Arnoldi basis, f, x, restart temporary
  if (pc && o.precond == 2) {  // block-tridiagonal factors: 3 level blocks per level, FP64 assembly batch
    const long long tz = D == 3 ? o.tile[2] : 1;
    const long long lm = nv * 2 * o.tile[0] * tz, nlev = std::max(1, o.tile[1] / 2);
    const long long ntiles = npts / std::max<long long>(1, o.tile[0] * o.tile[1] * tz);
    const long long per = nlev * 3 * lm * lm;
    b += ntiles * per * (o.precond_prec == 64 ? 16 : 8);
    b += std::min<long long>(ntiles, std::max<long long>(1, (1ll << 30) / (per * 16))) * per * 16;
    b += (long long)(nv + 1) * npts * 16;                // base fields for the reduced table
  } else if (pc) {
    const long long tz = D == 3 ? o.tile[2] : 1;
    const long long bsz = nv * o.tile[0] * o.tile[1] * tz;
    const long long ntiles = npts / std::max<long long>(1, o.tile[0] * o.tile[1] * tz);
    const long long bb = bsz * bsz;
    b += ntiles * bb * (o.precond_prec == 64 ? 16 : o.precond_prec == 32 ? 8 : 4);  // inverses
    const long long batch = std::min<long long>(ntiles, std::max<long long>(1, (1ll << 30) / (bb * 16)));
    b += batch * bb * 16;                                  // assembly batch
    if (o.precond_prec == 16) b += batch * bb * 8;         // FP32 inversion before rounding to BF16
    if (o.precond_factor && o.precond_prec != 64)          // pivots and the saved rows of the blocked sweep
      b += batch * bsz * (4 + (bsz <= 512 ? 128 : 256) * 8);
    const long long la = std::max<long long>({(long long)g->nx, (long long)g->ny, D == 3 ? g->nz : 1});
    b += (long long)D * 3 * la * la * 16;                  // 1-D derivative matrices
  }
  return b + b / 10 + (8ll << 20);                         // 10% and 8 MB for tables and alignment
}

// ---------------------------------------------------------------------------
// Batch
// ---------------------------------------------------------------------------
extern "C" stab_status stab_eigs_batch(stab_handle* hs, stab_eig_job* jobs, int count, int concurrency) {
  if (!hs || !jobs || count < 0) return STAB_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return STAB_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) {
        ((StabHandle*)hs[i])->err = "stab_eigs_batch: a handle appears twice";
        return STAB_ERR_INVALID_ARG;
      }
  }
  if (concurrency < 1) concurrency = count;
  concurrency = std::max(1, std::min(concurrency, count));
  // every handle on a private stream for the duration, ordered after its own stream
  std::vector<cudaStream_t> own(count, nullptr), priv(count, nullptr);
  stab_status first_err = STAB_OK;
  for (int i = 0; i < count; ++i) {
    StabHandle* h = (StabHandle*)hs[i];
    cudaSetDevice(h->device);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess ||
        cudaStreamCreateWithFlags(&priv[i], cudaStreamNonBlocking) != cudaSuccess) {
      h->err = "stab_eigs_batch: stream set-up failed";
      for (int j = 0; j <= i; ++j)
        if (priv[j]) cudaStreamDestroy(priv[j]);
      return STAB_ERR_CUDA;
    }
    own[i] = h->stream;
    h->stream = priv[i];
  }
  std::mutex mu;
  int next = 0;
  auto worker = [&]() {
    for (;;) {
      int i;
      {
        std::lock_guard<std::mutex> lk(mu);
        if (next >= count) return;
        i = next++;
      }
      StabHandle* h = (StabHandle*)hs[i];
      cudaSetDevice(h->device);
      stab_eig_job& J = jobs[i];
      J.nconv = 0;
      J.status = stab_eigs(hs[i], J.sigma_re, J.sigma_im, J.tau_re, J.tau_im, J.nev, J.ncv, J.tol, J.v0, J.lambda, J.vecs,
                           J.resid, &J.nconv, &J.stats);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < concurrency; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i) {
    StabHandle* h = (StabHandle*)hs[i];
    cudaSetDevice(h->device);
    cudaStreamSynchronize(priv[i]);
    h->stream = own[i];
    cudaStreamDestroy(priv[i]);
    if (jobs[i].status != STAB_OK && first_err == STAB_OK) first_err = jobs[i].status;
  }
  return first_err;
}

// ---------------------------------------------------------------------------
// Server
// ---------------------------------------------------------------------------
struct ServerReq {
  long long id = 0;
  std::vector<double> q0;
  stab_grid grid{};
  double Ma = 0, Re = 0, Pr = 0;
  stab_opts opts{};
  double sr = 0, si = 0, tr = 0, ti = 0, tol = 0;
  int nev = 0, ncv = 0;
  long long est = 0;
  void* vecs_host = nullptr;
  // results
  bool done = false;
  stab_status status = STAB_OK;
  int nconv = 0;
  std::vector<double> lambda, resid;
  stab_stats stats{};
  Clock::time_point t_submit, t_start, t_end;
  std::string err;
};

struct stab_server_s {
  int device = 0;
  int slots = 1;
  int cohort = 1;  // requests a worker takes at once and solves in lockstep (stab_jv_batch_eigs)
  long long budget = 0;
  int autotune = 0;
  std::mutex mu;
  std::condition_variable cv;      // workers: queue / memory changes
  std::condition_variable done_cv; // waiters: a request finished
  std::deque<ServerReq*> queue;
  std::map<long long, ServerReq*> reqs;
  long long next_id = 1;
  long long in_use = 0, peak_in_use = 0;
  int running = 0, peak_running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
};

namespace {

bool y_only(const std::vector<double>& q, const stab_grid& g, int nv) {
  const long long npts = (long long)g.nx * g.ny * g.nz;
  for (int v = 0; v < nv; ++v)
    for (int k = 0; k < g.nz; ++k)
      for (int j = 0; j < g.ny; ++j) {
        const double* row = q.data() + v * npts + ((long long)k * g.ny + j) * g.nx;
        const double ref = q[v * npts + (long long)j * g.nx];
        for (int i = 0; i < g.nx; ++i)
          if (row[i] != ref) return false;
      }
  return true;
}

void serve_one(stab_server_s* S, ServerReq* R, cudaStream_t st) {
  stab_handle h = nullptr;
  R->lambda.assign(2 * (size_t)R->nev, 0.0);
  R->resid.assign(R->nev, 0.0);
  stab_status s = stab_create(&h, R->q0.data(), 0, &R->grid, R->Ma, R->Re, R->Pr, &R->opts, st);
  if (s != STAB_OK) {
    R->status = s;
    R->err = stab_last_error(nullptr);
    return;
  }
  if (S->autotune) stab_autotune(h, 0, nullptr, nullptr);
  void* dvecs = nullptr;
  const size_t vbytes = (size_t)R->nev * stab_size(h) * 2 * sizeof(double);
  if (R->vecs_host && cudaMallocAsync(&dvecs, vbytes, st) != cudaSuccess) {
    R->status = STAB_ERR_OOM;
    R->err = "eigenvector buffer";
    stab_destroy(h);
    return;
  }
  R->status = stab_eigs(h, R->sr, R->si, R->tr, R->ti, R->nev, R->ncv, R->tol, nullptr, R->lambda.data(), dvecs,
                        R->resid.data(), &R->nconv, &R->stats);
  if (R->status != STAB_OK) R->err = stab_last_error(h);
  if (dvecs) {
    if (R->status == STAB_OK || R->status == STAB_ERR_NOT_CONVERGED)
      cudaMemcpyAsync(R->vecs_host, dvecs, vbytes, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dvecs, st);
    cudaStreamSynchronize(st);
  }
  stab_destroy(h);
}

// A cohort of requests taken at once by one worker: those whose handles can
// be batched (base flow varying in y only, FP64 GMRES basis, no LGMRES) are
// solved together by stab_jv_batch_eigs (every phase one launch for the
// cohort), the others one after the other.
void serve_cohort(stab_server_s* S, std::vector<ServerReq*>& C, cudaStream_t st) {
  if (C.size() == 1) {
    serve_one(S, C[0], st);
    return;
  }
  std::vector<stab_handle> hs(C.size(), nullptr);
  std::vector<void*> dvecs(C.size(), nullptr);
  std::vector<size_t> vbytes(C.size(), 0);
  std::vector<int> batched;
  for (size_t i = 0; i < C.size(); ++i) {
    ServerReq* R = C[i];
    R->lambda.assign(2 * (size_t)R->nev, 0.0);
    R->resid.assign(R->nev, 0.0);
    stab_status s = stab_create(&hs[i], R->q0.data(), 0, &R->grid, R->Ma, R->Re, R->Pr, &R->opts, st);
    if (s != STAB_OK) {
      R->status = s;
      R->err = stab_last_error(nullptr);
      hs[i] = nullptr;
      continue;
    }
    if (S->autotune) stab_autotune(hs[i], 0, nullptr, nullptr);
    vbytes[i] = (size_t)R->nev * stab_size(hs[i]) * 2 * sizeof(double);
    if (R->vecs_host && cudaMallocAsync(&dvecs[i], vbytes[i], st) != cudaSuccess) {
      R->status = STAB_ERR_OOM;
      R->err = "eigenvector buffer";
      dvecs[i] = nullptr;
      stab_destroy(hs[i]);
      hs[i] = nullptr;
      continue;
    }
    const StabHandle* h = (const StabHandle*)hs[i];
    if (h->homog && h->d_coef && !h->force_dn_path && h->opts.gmres_basis_prec == 64 && h->opts.lgmres_k == 0 &&
        h->opts.gmres_inner_m == 0 && h->opts.precond != 2)
      batched.push_back((int)i);
  }
  if (batched.size() >= 2) {
    std::vector<stab_handle> bh;
    std::vector<stab_eig_job> jobs(batched.size());
    for (size_t q = 0; q < batched.size(); ++q) {
      const int i = batched[q];
      ServerReq* R = C[i];
      bh.push_back(hs[i]);
      stab_eig_job& J = jobs[q];
      std::memset(&J, 0, sizeof(J));
      J.sigma_re = R->sr; J.sigma_im = R->si; J.tau_re = R->tr; J.tau_im = R->ti;
      J.nev = R->nev; J.ncv = R->ncv; J.tol = R->tol;
      J.lambda = R->lambda.data();
      J.resid = R->resid.data();
      J.vecs = dvecs[i];
    }
    stab_jv_batch B = nullptr;
    stab_status s = stab_jv_batch_create(&B, bh.data(), (int)bh.size(), st);
    if (s == STAB_OK) {
      stab_jv_batch_eigs(B, jobs.data());
      const std::string msg = stab_jv_batch_last_error(B);
      stab_jv_batch_destroy(B);
      for (size_t q = 0; q < batched.size(); ++q) {
        ServerReq* R = C[batched[q]];
        R->status = jobs[q].status;
        R->nconv = jobs[q].nconv;
        R->stats = jobs[q].stats;
        if (R->status != STAB_OK) R->err = msg;
      }
    } else {
      batched.clear();  // solved one by one below
    }
  } else {
    batched.clear();
  }
  for (size_t i = 0; i < C.size(); ++i) {
    ServerReq* R = C[i];
    if (!hs[i]) continue;
    if (std::find(batched.begin(), batched.end(), (int)i) == batched.end()) {
      R->status = stab_eigs(hs[i], R->sr, R->si, R->tr, R->ti, R->nev, R->ncv, R->tol, nullptr, R->lambda.data(),
                            dvecs[i], R->resid.data(), &R->nconv, &R->stats);
      if (R->status != STAB_OK) R->err = stab_last_error(hs[i]);
    }
    if (dvecs[i]) {
      if (R->status == STAB_OK || R->status == STAB_ERR_NOT_CONVERGED)
        cudaMemcpyAsync(R->vecs_host, dvecs[i], vbytes[i], cudaMemcpyDeviceToHost, st);
      cudaFreeAsync(dvecs[i], st);
    }
  }
  cudaStreamSynchronize(st);
  for (stab_handle h : hs)
    if (h) stab_destroy(h);
}

void worker_main(stab_server_s* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    std::vector<ServerReq*> C;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // admission: first come, first served; the head waits until its memory fits, then (cohort > 1)
      // the requests queued behind it join while their memory fits
      S->cv.wait(lk, [&] { return S->stop || (!S->queue.empty() && S->in_use + S->queue.front()->est <= S->budget); });
      if (S->stop) break;  // stab_server_destroy has emptied the queue
      do {
        ServerReq* R = S->queue.front();
        S->queue.pop_front();
        S->in_use += R->est;
        S->running++;
        R->t_start = Clock::now();
        C.push_back(R);
      } while ((int)C.size() < S->cohort && !S->queue.empty() && S->in_use + S->queue.front()->est <= S->budget);
      S->peak_in_use = std::max(S->peak_in_use, S->in_use);
      S->peak_running = std::max(S->peak_running, S->running);
    }
    serve_cohort(S, C, st);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (ServerReq* R : C) {
        R->t_end = Clock::now();
        R->done = true;
        S->in_use -= R->est;
        S->running--;
      }
    }
    S->cv.notify_all();
    S->done_cv.notify_all();
  }
  cudaStreamDestroy(st);
}

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

}  // namespace

extern "C" stab_status stab_server_create(stab_server* out, int slots, long long mem_budget_bytes, int autotune) {
  if (!out || slots < 1 || slots > 256 || mem_budget_bytes <= 0) return STAB_ERR_INVALID_ARG;
  *out = nullptr;
  stab_server_s* S = new (std::nothrow) stab_server_s;
  if (!S) return STAB_ERR_OOM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return STAB_ERR_CUDA;
  }
  S->slots = slots;
  S->budget = mem_budget_bytes;
  S->autotune = autotune;
  for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return STAB_OK;
}

extern "C" stab_status stab_server_set_cohort(stab_server S, int cohort) {
  if (!S || cohort < 1 || cohort > 4096) return STAB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  S->cohort = cohort;
  return STAB_OK;
}

extern "C" stab_status stab_server_submit(stab_server S, const stab_request* q, long long* id) {
  if (!S || !q || !id || !q->base_flow) return STAB_ERR_INVALID_ARG;
  const stab_grid& g = q->grid;
  if (g.dim < 2 || g.dim > 3 || g.nx < 1 || g.ny < 1 || g.nz < 1 || q->nev < 1 || q->ncv <= q->nev) return STAB_ERR_INVALID_ARG;
  ServerReq* R = new (std::nothrow) ServerReq;
  if (!R) return STAB_ERR_OOM;
  const long long n = (long long)(g.dim + 2) * g.nx * g.ny * g.nz;
  R->q0.assign(q->base_flow, q->base_flow + n);
  R->grid = g;
  R->Ma = q->Ma;
  R->Re = q->Re;
  R->Pr = q->Pr;
  if (q->opts) R->opts = *q->opts;
  else stab_default_opts(&R->opts);
  R->sr = q->sigma_re;
  R->si = q->sigma_im;
  R->tr = q->tau_re;
  R->ti = q->tau_im;
  R->nev = q->nev;
  R->ncv = q->ncv;
  R->tol = q->tol;
  R->vecs_host = q->vecs;
  R->est = stab_estimate_bytes(&g, &R->opts, y_only(R->q0, g, g.dim + 2), q->nev, q->ncv) +
           (q->vecs ? (long long)q->nev * n * 16 : 0);
  R->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (R->est > S->budget) {
      delete R;
      return STAB_ERR_OOM;
    }
    R->id = S->next_id++;
    S->reqs[R->id] = R;
    S->queue.push_back(R);
    *id = R->id;
  }
  S->cv.notify_all();
  return STAB_OK;
}

extern "C" stab_status stab_server_wait(stab_server S, long long id, double timeout_s) {
  if (!S) return STAB_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return STAB_ERR_INVALID_ARG;
  ServerReq* R = it->second;
  if (timeout_s < 0) S->done_cv.wait(lk, [&] { return R->done; });
  else S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return R->done; });
  return R->done ? STAB_OK : STAB_ERR_TIMEOUT;
}

extern "C" stab_status stab_server_result(stab_server S, long long id, double* lambda, double* resid,
                                          stab_request_info* info) {
  if (!S) return STAB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return STAB_ERR_INVALID_ARG;
  ServerReq* R = it->second;
  if (!R->done) return STAB_ERR_BUSY;
  if (lambda) std::memcpy(lambda, R->lambda.data(), R->lambda.size() * sizeof(double));
  if (resid) std::memcpy(resid, R->resid.data(), R->resid.size() * sizeof(double));
  if (info) {
    info->status = R->status;
    info->nconv = R->nconv;
    info->queued_s = secs(R->t_submit, R->t_start);
    info->run_s = secs(R->t_start, R->t_end);
    info->latency_s = secs(R->t_submit, R->t_end);
    info->est_bytes = R->est;
    info->stats = R->stats;
  }
  S->reqs.erase(it);
  delete R;
  return STAB_OK;
}

extern "C" stab_status stab_server_stats(stab_server S, long long* peak_bytes, int* peak_running, int* queued,
                                         int* running) {
  if (!S) return STAB_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  if (peak_bytes) *peak_bytes = S->peak_in_use;
  if (peak_running) *peak_running = S->peak_running;
  if (queued) *queued = (int)S->queue.size();
  if (running) *running = S->running;
  return STAB_OK;
}

extern "C" void stab_server_destroy(stab_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (ServerReq* R : S->queue) {  // never started
      R->status = STAB_ERR_BUSY;
      R->err = "server destroyed before the request started";
      R->done = true;
    }
    S->queue.clear();
  }
  S->cv.notify_all();
  S->done_cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}
