// Host side of the C ABI declared in include/domdec.h: handle lifetime, the
// partitions and staggered sub-batches (Section 5.3), the sweep driver
// (Algorithm 2 over Algorithm 4 per sub-batch),
// and the read-back entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dd_common.cuh"
#include "domdec.h"

// ---- kernels' launch wrappers (dd_cell.cu, dd_sweep.cu, dd_sinkhorn.cu)
size_t cell_smem_bytes(int s, int cap_side, int cap_ny, int precision);
cudaError_t launch_cell_solve(const DevState& S, const CellDesc* cells, const int* order, const int* nbig_p,
                              int begin, int nbatch, int precision, size_t smem, int nctas, int crun, int cluster,
                              cudaStream_t st);
cudaError_t launch_cell_order(const DevState& S, int part, int mode, int slots, int C, double factor,
                              cudaStream_t st);
size_t dist_smem_bytes(int s, int C, int cap_w, int cap_hl, int cap_nyl, int precision);
int cell_static_smem(int precision);
int cell_resident_ctas(size_t smem, int C, int precision);
cudaError_t launch_cell_solve_multi(const DevState* states, const CellRef* refs, int nref, int part, int* order,
                                    int* nbig, unsigned int* queue, size_t smem, int precision, int C,
                                    double factor, int nctas, cudaStream_t st);
int cell_multi_resident_ctas(size_t smem, int C, int precision);
cudaError_t launch_decide_multi(const DevState* states, int ninst, int maxn, int part, int sub, cudaStream_t st);
cudaError_t launch_apply_multi(const DevState* states, const CellRef* refs, int nref, int part, cudaStream_t st);
cudaError_t launch_compact_multi(const DevState* states, int ninst, int max_nbasic, cudaStream_t st);
cudaError_t launch_decide(const DevState& S, const CellDesc* cells, int begin, int nbatch, cudaStream_t st);
cudaError_t launch_line_search(const DevState& S, const CellDesc* cells, int begin, int nbatch, double* partials,
                               cudaStream_t st);
cudaError_t launch_apply(const DevState& S, const CellDesc* cells, int begin, int nbatch, cudaStream_t st);
cudaError_t launch_compact(const DevState& S, long long* newoff, cudaStream_t st);
cudaError_t launch_prepare_inputs(const double* mu, const double* nu, double* logmu, double* lognu, int n,
                                  int* status, cudaStream_t st);
cudaError_t launch_init_product_boxes(const DevState& S, double* nu_mom, double* mumass, long long* newoff,
                                      cudaStream_t st);
cudaError_t launch_init_product_fill(const DevState& S, double* nu_mom, double* mumass, long long* newoff,
                                     cudaStream_t st);
cudaError_t launch_init_duals_boxes(const DevState& S, const double* alpha0, const double* beta0, double eps0,
                                    double* nu_mom, double* mumass, long long* newoff, float* gscratch,
                                    cudaStream_t st);
cudaError_t launch_init_duals_fill(const DevState& S, const double* alpha0, const double* beta0, double eps0,
                                   const double* w, long long* newoff, cudaStream_t st);
cudaError_t launch_score(const DevState& S, double* out, cudaStream_t st, double* partials);
cudaError_t launch_cert(const DevState& S, const double* z, double* beta_out, double* out, cudaStream_t st,
                        double* partials);
cudaError_t launch_regrow(const DevState& S, double* new0, double* new1, long long* newoff, cudaStream_t st);
cudaError_t global_lse64(const double* pot, const double* logm, double eps, double h, int N, double* out,
                         double* buf_a, double* buf_b, double* buf_c, cudaStream_t st);
int full_sinkhorn_dev(const double* mu, const double* nu, const double* logmu, const double* lognu, int N,
                      double eps_start, double eps, double lam, int variant, int precision, int maxit,
                      double err, int check_every, double* alpha, double* beta, double* out, double* d_eval,
                      cudaStream_t st, cudaError_t* cerr);
size_t adjoint_scratch_size(int N, int precision);
cudaError_t adjoint_dev(const double* mu, const double* nu, const double* alpha, const double* beta, int N,
                        double eps, double lam, int precision, double* grad_mu, double* grad_nu, double* grad_x,
                        double* d_out, void* scratch, int* d_bad, cudaStream_t st);

namespace {
constexpr int LOGCAP = 4096;
constexpr int NCOUNT = 9;
}  // namespace

struct domdec_s {
  domdec_params p;
  int N = 0, s = 0, nb = 0, nbasic = 0, n = 0;
  cudaStream_t st = nullptr;
  DevState S;
  std::vector<void*> allocs;
  CellDesc* d_cells[2] = {nullptr, nullptr};
  int sub_start[2][5];
  int ncell[2] = {0, 0};
  int max_batch = 0;
  long long* d_newoff = nullptr;
  double* d_scratch = nullptr;  // 64 doubles
  double* d_partials = nullptr; // kRedBlocks * 8 doubles: block partials of the grid reductions
  double* d_numom = nullptr;
  double* d_mumass = nullptr;
  double* h_pinned = nullptr;   // 64 doubles
  long long sweeps = 0;
  long long slot = 0;
  unsigned long long maxit_seen = 0;  // maxit-cell counter at the previous domdec_sync
  long long arena_regrows = 0;        // arena growths after a halted sub-batch
  long long regroups = 0;             // switches to the largest cluster after a halted sweep
  int sticky = 0;
  int last_batch = 0;
  double eps0 = 0.0, err0 = 0.0;           // eps and err given at domdec_init (restored by domdec_reset)
  double *d_a0 = nullptr, *d_b0 = nullptr, *d_w4 = nullptr;  // warm-start duals and 4 N*N scratch
  int res[4] = {0, 0, 0, 0};   // resident CTAs of the cell kernel with clusters of 1, 2, 4, 8
  int crun = 1;            // cluster size of the cell launches (<= S.dist_c)
  double split = 2.0;      // cluster cells: work above split x the mean work per CTA
  int cell_nctas = 0;      // persistent CTAs of the cell kernel (whole clusters of crun)
  int helper_ctas = 0;     // single CTAs on the SMs that the resident clusters leave idle
  cudaStream_t st2 = nullptr;               // their stream, forked from and joined to st per sub-batch
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t cell_smem = 0;    // its dynamic shared memory
  int order_mode = 0;      // k_cell_order: 0 automatic, 1 every fitting cell on a cluster, 2 none
  // profiling: pending event pairs per kernel class
  struct EvPair { cudaEvent_t a, b; int cls; };
  std::vector<EvPair> pend;
  std::vector<cudaEvent_t> pool;
  double kt[4] = {0, 0, 0, 0};
  long long kn[4] = {0, 0, 0, 0};
};

namespace {

int fail(domdec_s* h, int code) {
  if (h && code < 0) h->sticky = code;
  return code;
}

template <typename T>
cudaError_t dalloc(domdec_s* h, T** ptr, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *ptr = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

void build_partition(domdec_s* h, int which, std::vector<CellDesc>& out, int* sub_start) {
  const int s = h->s, nb = h->nb, N = h->N, off = which;
  const int nc = nb / 2 + off;
  std::vector<CellDesc> subs[4];
  for (int P = 0; P < nc; ++P)
    for (int Q = 0; Q < nc; ++Q) {
      const int lb1 = 2 * P - off, lb2 = 2 * Q - off;
      CellDesc cd;
      const int xlo1 = std::max(0, s * lb1), xhi1 = std::min(N, s * (lb1 + 2));
      const int xlo2 = std::max(0, s * lb2), xhi2 = std::min(N, s * (lb2 + 2));
      cd.i0 = xlo1; cd.j0 = xlo2; cd.nx1 = xhi1 - xlo1; cd.nx2 = xhi2 - xlo2;
      for (int q = 0; q < 4; ++q) cd.mem[q] = -1;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const int I = lb1 + a, J = lb2 + b;
          if (I < 0 || J < 0 || I >= nb || J >= nb) continue;
          // quadrant relative to the X box origin
          const int qr = (I * s - xlo1) >= s ? 1 : 0, qc = (J * s - xlo2) >= s ? 1 : 0;
          cd.mem[2 * qr + qc] = I * nb + J;
        }
      subs[2 * (P % 2) + (Q % 2)].push_back(cd);
    }
  out.clear();
  sub_start[0] = 0;
  for (int b = 0; b < 4; ++b) {
    out.insert(out.end(), subs[b].begin(), subs[b].end());
    sub_start[b + 1] = (int)out.size();
  }
}

int check_params(const domdec_params* p, int N) {
  if (!p || N <= 0) return DOMDEC_EINVAL;
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return DOMDEC_EINVAL;
  if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return DOMDEC_EINVAL;
  if (p->basic_cell < 1 || p->basic_cell > 16 || N % (2 * p->basic_cell)) return DOMDEC_EINVAL;
  if (p->maxit < 1 || p->newton_maxit < 1) return DOMDEC_EINVAL;
  if (p->strategy < 0 || p->strategy > 5 || (p->precision != 0 && p->precision != 1)) return DOMDEC_EINVAL;
  if (!(p->trunc_thr >= 0.0) || p->box_margin < 0) return DOMDEC_EINVAL;
  if ((p->cell_ctas != 0 && p->cell_ctas != 1 && p->cell_ctas != 2 && p->cell_ctas != 4 && p->cell_ctas != 8) ||
      p->cell_ti < 0 || p->cell_ti > 1)
    return DOMDEC_EINVAL;
  if (p->balance < 0 || p->balance > 1) return DOMDEC_EINVAL;
  if (!(p->cell_split >= 0.0) || std::isinf(p->cell_split)) return DOMDEC_EINVAL;
  return DOMDEC_OK;
}

int enqueue_sweep(domdec_s* h, int part, long long slot0, int first);
int batches_per_sweep(domdec_s* h, int part);
int recover_halt(domdec_s* h, int st);
void set_cluster(domdec_s* h, int C);

int read_status(domdec_s* h) {
  // slot 63 of the pinned buffer is reserved for the status word
  int* hs = reinterpret_cast<int*>(h->h_pinned + 63);
  int st = 0;
  for (int attempt = 0;; ++attempt) {
    cudaError_t e = cudaMemcpyAsync(hs, h->S.status, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
    st = *hs;
    if (st != ST_ARENA && st != ST_REGROUP) break;
    // halted sweeps: a sub-batch's new boxes did not fit (grow the arena) or a
    // cell needs a larger cluster (switch to the layout's largest); then rerun
    // what did not run
    if (attempt >= 4) return fail(h, st == ST_ARENA ? DOMDEC_EARENA : DOMDEC_ETOOBIG);
    const int rc = recover_halt(h, st);
    if (rc) return fail(h, rc);
  }
  if (st & ST_BADINPUT) return fail(h, DOMDEC_EINVAL);
  if (st & ST_TOOBIG) return fail(h, DOMDEC_ETOOBIG);
  if (st & (ST_ARENA | ST_ARENA_LOST)) return fail(h, DOMDEC_EARENA);
  if (st & ST_EMPTY) return fail(h, DOMDEC_EEMPTY);
  if (st & ST_NONFINITE) return fail(h, DOMDEC_ENONFINITE);
  return DOMDEC_OK;
}

// Make sure each arena has room for 4x the live data (at a synchronisation point).
int ensure_arena(domdec_s* h) {
  unsigned long long live = 0;
  cudaError_t e = cudaMemcpyAsync(&live, h->S.head, sizeof(live), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  if ((long long)live * 4 <= h->S.cap) return DOMDEC_OK;
  long long ncap = (long long)live * 8;
  double *a0 = nullptr, *a1 = nullptr;
  if (cudaMalloc(&a0, ncap * sizeof(double)) != cudaSuccess) return fail(h, DOMDEC_ENOMEM);
  if (cudaMalloc(&a1, ncap * sizeof(double)) != cudaSuccess) { cudaFree(a0); return fail(h, DOMDEC_ENOMEM); }
  if (launch_regrow(h->S, a0, a1, h->d_newoff, h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  for (auto& q : h->allocs)
    if (q == h->S.arena[0] || q == h->S.arena[1]) { cudaFree(q); q = nullptr; }
  h->allocs.push_back(a0);
  h->allocs.push_back(a1);
  h->S.arena[0] = a0;
  h->S.arena[1] = a1;
  h->S.cap = ncap;
  return DOMDEC_OK;
}

// Resume a handle whose enqueued sweeps halted (the state is that after the
// last completed sub-batch): ST_ARENA (the reservation of k_decide) grows the
// arena, ST_REGROUP (k_cell_order) switches the cell launches to the layout's
// largest cluster size; then the halt is cleared and the sub-batches that did
// not run are enqueued again -- the device's decision count says how many of
// the enqueued sub-batches completed.
int recover_halt(domdec_s* h, int st) {
  unsigned long long done = 0, live = 0;
  cudaError_t e = cudaMemcpyAsync(&done, h->S.slotctr, sizeof(done), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&live, h->S.head, sizeof(live), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  if (st == ST_REGROUP) {
    set_cluster(h, h->S.dist_c);
    ++h->regroups;
  } else {
    const long long ncap = std::max(2 * h->S.cap, 4 * (long long)live + 1024);
    double *a0 = nullptr, *a1 = nullptr;
    if (cudaMalloc(&a0, ncap * sizeof(double)) != cudaSuccess) return DOMDEC_ENOMEM;
    if (cudaMalloc(&a1, ncap * sizeof(double)) != cudaSuccess) { cudaFree(a0); return DOMDEC_ENOMEM; }
    if (launch_regrow(h->S, a0, a1, h->d_newoff, h->st) != cudaSuccess) return DOMDEC_ECUDA;
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return DOMDEC_ECUDA;
    for (auto& q : h->allocs)
      if (q == h->S.arena[0] || q == h->S.arena[1]) { cudaFree(q); q = nullptr; }
    h->allocs.push_back(a0);
    h->allocs.push_back(a1);
    h->S.arena[0] = a0;
    h->S.arena[1] = a1;
    h->S.cap = ncap;
    ++h->arena_regrows;
  }
  if (cudaMemsetAsync(h->S.status, 0, sizeof(int), h->st) != cudaSuccess) return DOMDEC_ECUDA;
  // the enqueued sweeps, oldest first: find the first sub-batch that did not run
  long long cum = 0;
  for (long long k = 0; k < h->sweeps; ++k) {
    const int part = (int)(k % 2);
    const int nb = batches_per_sweep(h, part);
    if ((unsigned long long)(cum + nb) > done) {
      const int first = (int)((long long)done - cum);
      int rc = enqueue_sweep(h, part, cum, first);
      long long c2 = cum + nb;
      for (long long k2 = k + 1; rc == DOMDEC_OK && k2 < h->sweeps; ++k2) {
        rc = enqueue_sweep(h, (int)(k2 % 2), c2, 0);
        c2 += batches_per_sweep(h, (int)(k2 % 2));
      }
      return rc;
    }
    cum += nb;
  }
  return DOMDEC_OK;
}

cudaEvent_t take_event(domdec_s* h) {
  if (!h->pool.empty()) {
    cudaEvent_t e = h->pool.back();
    h->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Record a start event (profiling only); returns it, or nullptr.
cudaEvent_t prof_begin(domdec_s* h) {
  if (!h->p.profile) return nullptr;
  cudaEvent_t a = take_event(h);
  cudaEventRecord(a, h->st);
  return a;
}

void prof_end(domdec_s* h, cudaEvent_t a, int cls) {
  if (!a) return;
  cudaEvent_t b = take_event(h);
  cudaEventRecord(b, h->st);
  h->pend.push_back({a, b, cls});
}

// Fold finished event pairs into the accumulators (after a synchronisation).
void prof_collect(domdec_s* h) {
  for (auto& ev : h->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) {
      h->kt[ev.cls] += ms;
      h->kn[ev.cls] += 1;
    }
    h->pool.push_back(ev.a);
    h->pool.push_back(ev.b);
  }
  h->pend.clear();
}

// Cluster size of the cell launches: C (1, 2, 4, 8; at most the layout's
// dist_c, and only if such clusters are resident), the grid size, and the
// helper grid on the SMs the clusters leave idle.
void set_cluster(domdec_s* h, int C) {
  int ci = 0;
  while ((1 << ci) < C && ci < 3) ++ci;
  C = 1 << ci;
  if (C > std::max(1, h->S.dist_c) || h->res[ci] < C) {
    C = 1;
    ci = 0;
  }
  h->crun = C;
  h->cell_nctas = std::max(C, h->res[ci] / C * C);
  h->helper_ctas = C > 1 && h->st2 ? std::max(0, h->res[0] - h->cell_nctas) : 0;
}

// Enqueue one sweep of partition `part`, from its `first`-th non-empty batch on
// (0: the whole sweep).
int enqueue_sweep(domdec_s* h, int part, long long slot0, int first = 0) {
  const int prec = h->p.precision;
  std::vector<std::pair<int, int>> batches;
  if (h->p.strategy == DOMDEC_STAGGERED || h->p.strategy == DOMDEC_STAGGERED_LINE) {
    for (int b = 0; b < 4; ++b) batches.push_back({h->sub_start[part][b], h->sub_start[part][b + 1]});
  } else {
    batches.push_back({0, h->ncell[part]});
  }
  int k = 0;
  // largest-first order of the cells of every sub-batch of this sweep (the
  // member boxes of a sub-batch do not change before its own cell solve)
  if (launch_cell_order(h->S, part, h->crun > 1 ? h->order_mode : 2, h->cell_nctas, h->crun, h->split, h->st) !=
      cudaSuccess)
    return DOMDEC_ECUDA;
  int nonempty = 0;
  for (auto& bt : batches) {
    const int begin = bt.first, nbt = bt.second - bt.first;
    if (nbt <= 0) continue;
    if (nonempty++ < first) continue;
    const int slot = (int)((slot0 + k++) % LOGCAP);
    (void)slot;
    cudaEvent_t ev = prof_begin(h);
    const int sub = (int)(&bt - batches.data());
    const int* nbig_p = h->S.nbig + part * 4 + (batches.size() == 4 ? sub : 0);
    const int C = h->crun;
    if (launch_cell_solve(h->S, h->d_cells[part], h->S.order[part], nbig_p, begin, nbt, prec, h->cell_smem,
                          h->cell_nctas, C, C, h->st) != cudaSuccess)
      return DOMDEC_ECUDA;
    if (h->helper_ctas > 0) {
      // single CTAs on the SMs left idle by the clusters, same phase-2 queue
      if (cudaEventRecord(h->ev_fork, h->st) != cudaSuccess || cudaStreamWaitEvent(h->st2, h->ev_fork, 0) != cudaSuccess ||
          launch_cell_solve(h->S, h->d_cells[part], h->S.order[part], nbig_p, begin, nbt, prec, h->cell_smem,
                            h->helper_ctas, C, 1, h->st2) != cudaSuccess ||
          cudaEventRecord(h->ev_join, h->st2) != cudaSuccess || cudaStreamWaitEvent(h->st, h->ev_join, 0) != cudaSuccess)
        return DOMDEC_ECUDA;
    }
    prof_end(h, ev, 0);
    ev = prof_begin(h);
    if (launch_decide(h->S, h->d_cells[part], begin, nbt, h->st) != cudaSuccess) return DOMDEC_ECUDA;
    if ((h->p.strategy == DOMDEC_LINE || h->p.strategy == DOMDEC_STAGGERED_LINE) &&
        launch_line_search(h->S, h->d_cells[part], begin, nbt, h->d_partials, h->st) != cudaSuccess)
      return DOMDEC_ECUDA;
    prof_end(h, ev, 1);
    ev = prof_begin(h);
    if (launch_apply(h->S, h->d_cells[part], begin, nbt, h->st) != cudaSuccess) return DOMDEC_ECUDA;
    prof_end(h, ev, 2);
    h->last_batch = nbt;
  }
  cudaEvent_t ev = prof_begin(h);
  if (launch_compact(h->S, h->d_newoff, h->st) != cudaSuccess) return DOMDEC_ECUDA;
  prof_end(h, ev, 3);
  return DOMDEC_OK;
}

// Copy mu, nu (and the warm-start duals) into the handle's buffers, clear the
// sweep state and build the initial plan (Algorithm 2, pi_init): the product
// plan, or exp((alpha0 + beta0 - c)/eps0) mu x nu.  Allocates only what does
// not exist yet (the arenas on the first call or when the new plan does not
// fit them, the dual buffers on the first call with duals).  Synchronises.
int load_problem(domdec_s* h, const double* mu, const double* nu, const double* alpha0, const double* beta0,
                 double eps0) {
  DevState& S = h->S;
  const int n = h->n, N = h->N;
  cudaStream_t st = h->st;
  cudaError_t e = cudaMemcpyAsync(const_cast<double*>(S.mu), mu, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(const_cast<double*>(S.nu), nu, n * sizeof(double), cudaMemcpyDefault, st);
  cudaMemsetAsync(S.status, 0, sizeof(int), st);
  cudaMemsetAsync(S.cur, 0, sizeof(int), st);
  cudaMemsetAsync(S.head, 0, sizeof(unsigned long long), st);
  cudaMemsetAsync(S.counters, 0, NCOUNT * sizeof(unsigned long long), st);
  cudaMemsetAsync(S.red_count, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(S.queue, 0, 2 * sizeof(unsigned int), st);
  cudaMemsetAsync(S.nbig, 0, 8 * sizeof(int), st);
  cudaMemsetAsync(S.spill_count, 0, sizeof(unsigned int), st);
  cudaMemsetAsync(S.dPY, 0, n * sizeof(double), st);
  cudaMemsetAsync(S.PY, 0, n * sizeof(double), st);
  cudaMemsetAsync(S.theta, 0, sizeof(double), st);
  cudaMemsetAsync(S.declog, 0, 4 * LOGCAP * sizeof(double), st);
  cudaMemsetAsync(S.slotctr, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = launch_prepare_inputs(S.mu, S.nu, const_cast<double*>(S.logmu), const_cast<double*>(S.lognu), n, S.status,
                              st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  if (alpha0 && !h->d_a0) {
    if (dalloc(h, &h->d_a0, n) != cudaSuccess || dalloc(h, &h->d_b0, n) != cudaSuccess ||
        dalloc(h, &h->d_w4, 4 * (size_t)n) != cudaSuccess)
      return DOMDEC_ENOMEM;
  }
  double *ad = h->d_a0, *bd = h->d_b0, *wtmp = h->d_w4;
  if (alpha0) {
    e = cudaMemcpyAsync(ad, alpha0, n * sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bd, beta0, n * sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
      e = launch_init_duals_boxes(S, ad, bd, eps0, h->d_numom, h->d_mumass, h->d_newoff,
                                  reinterpret_cast<float*>(wtmp), st);
  } else {
    e = launch_init_product_boxes(S, h->d_numom, h->d_mumass, h->d_newoff, st);
  }
  long long total = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, h->d_newoff + h->nbasic, sizeof(long long), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  int rc = read_status(h);
  if (rc) return rc;
  // default: 48 N^2 and at least 8x the initial plan; an explicit arena_factor is
  // taken as given (down to the initial plan itself: growth happens on demand)
  const double fac = h->p.arena_factor > 0 ? h->p.arena_factor : 48.0;
  const long long floor_cap = h->p.arena_factor > 0 ? total + 1024 : 8 * total + 1024;
  const long long need = std::max((long long)(fac * n), floor_cap);
  if (!S.arena[0] || S.cap < floor_cap) {
    for (auto& q : h->allocs)
      if (q && (q == S.arena[0] || q == S.arena[1])) { cudaFree(q); q = nullptr; }
    S.arena[0] = S.arena[1] = nullptr;
    if (dalloc(h, &S.arena[0], need) != cudaSuccess || dalloc(h, &S.arena[1], need) != cudaSuccess)
      return DOMDEC_ENOMEM;
    S.cap = need;
  }
  if (alpha0) {
    // w(x) = log sum_y exp(beta0/eps0 + log nu - c/eps0): P_X of the initial plan
    e = global_lse64(bd, S.lognu, eps0, 1.0 / N, N, wtmp, wtmp + n, wtmp + 2 * (size_t)n, wtmp + 3 * (size_t)n, st);
    if (e == cudaSuccess) e = launch_init_duals_fill(S, ad, bd, eps0, wtmp, h->d_newoff, st);
  } else {
    e = launch_init_product_fill(S, h->d_numom, h->d_mumass, h->d_newoff, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  rc = read_status(h);
  if (rc) return rc;
  h->sweeps = 0;
  h->slot = 0;
  h->maxit_seen = 0;
  h->last_batch = 0;
  for (int k = 0; k < 4; ++k) { h->kt[k] = 0.0; h->kn[k] = 0; }
  return DOMDEC_OK;
}

int batches_per_sweep(domdec_s* h, int part) {
  if (h->p.strategy != DOMDEC_STAGGERED && h->p.strategy != DOMDEC_STAGGERED_LINE)
    return h->ncell[part] > 0 ? 1 : 0;
  int c = 0;
  for (int b = 0; b < 4; ++b) c += h->sub_start[part][b + 1] > h->sub_start[part][b];
  return c;
}

}  // namespace

extern "C" {

void domdec_default_params(domdec_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps = 1.0;
  p->lambda = 1.0;
  p->basic_cell = 4;
  p->err = 2e-5;
  p->trunc_thr = 1e-15;
  p->tau = 0.0;
  p->strategy = DOMDEC_STAGGERED;
  p->maxit = 2000;
  p->newton_maxit = 30;
  p->precision = DOMDEC_FP32;
  p->box_margin = 0;
  p->max_ny = 0;
  p->arena_factor = 0.0;
  p->eps_init = 0.0;
}

const char* domdec_error_string(int code) {
  switch (code) {
    case DOMDEC_OK: return "ok";
    case DOMDEC_WNOTCONV: return "warning: some cell solves stopped at maxit";
    case DOMDEC_EINVAL: return "invalid argument";
    case DOMDEC_ENOMEM: return "device allocation failed";
    case DOMDEC_ECUDA: return "CUDA runtime error";
    case DOMDEC_ETOOBIG: return "a cell Y-box exceeds the kernel's shared-memory capacity (max_ny)";
    case DOMDEC_EARENA: return "box arena overflow";
    case DOMDEC_ESTATE: return "handle is in an error state";
    case DOMDEC_ENOLIB: return "library not loaded";
    case DOMDEC_EEMPTY: return "a composite cell has no Y-support left after truncation";
    case DOMDEC_ENONFINITE: return "a cell solve produced a non-finite value";
    default: return "unknown error";
  }
}

void domdec_free(domdec_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  prof_collect(h);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  if (h->st2) { cudaStreamSynchronize(h->st2); cudaStreamDestroy(h->st2); }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (void* q : h->allocs)
    if (q) cudaFree(q);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  delete h;
}

int domdec_init(domdec_t* out, const double* mu, const double* nu, int N, const domdec_params* pin,
                const double* alpha0, const double* beta0, void* stream) {
  if (!out) return DOMDEC_EINVAL;
  *out = nullptr;
  if (!mu || !nu) return DOMDEC_EINVAL;
  int rc = check_params(pin, N);
  if (rc) return rc;
  if ((alpha0 == nullptr) != (beta0 == nullptr)) return DOMDEC_EINVAL;
  if (alpha0 && !(pin->eps_init > 0.0)) return DOMDEC_EINVAL;
  domdec_s* h = new (std::nothrow) domdec_s();
  if (!h) return DOMDEC_ENOMEM;
  h->p = *pin;
  h->N = N; h->s = pin->basic_cell; h->nb = N / h->s; h->nbasic = h->nb * h->nb; h->n = N * N;
  h->st = reinterpret_cast<cudaStream_t>(stream);
  const int n = h->n;
  DevState& S = h->S;
  std::memset(&S, 0, sizeof(S));
  S.N = N; S.s = h->s; S.nb = h->nb; S.nbasic = h->nbasic;
  S.h = 1.0 / N; S.eps = pin->eps; S.lam = pin->lambda; S.thr = pin->trunc_thr; S.err = pin->err;
  S.ti = pin->cell_ti ? 1 : 0;
  S.balance = pin->balance ? 1 : 0;
  S.tau = pin->tau; S.maxit = pin->maxit; S.newton_maxit = pin->newton_maxit; S.strategy = pin->strategy;
  S.margin = pin->box_margin;
  // shared-memory capacity of the cell kernel
  int dev = 0, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // dynamic shared memory left beside the kernels' static shared memory
  const int smem_budget = smem_optin - cell_static_smem(pin->precision) - 64;
  int cap_ny = pin->max_ny > 0 ? pin->max_ny : (pin->precision ? 3072 : 8192);
  int cap_side = std::min(N, 128);
  for (;;) {
    cap_side = std::min(cap_side, cap_ny);
    // epilogue scratch (3 nx1 W) must fit in the T/U/bl/lrho/Zv region
    while (2 * h->s * cap_side > 3 * cap_ny && cap_side > 1) --cap_side;
    if (cell_smem_bytes(h->s, cap_side, cap_ny, pin->precision) <= (size_t)smem_budget || cap_ny <= 64) break;
    cap_ny -= 256;
  }
  S.cap_ny = cap_ny;
  S.cap_side = cap_side;
  if (cell_smem_bytes(h->s, cap_side, cap_ny, pin->precision) > (size_t)smem_budget) {
    delete h;
    return DOMDEC_EINVAL;
  }
  // clusters for the largest cells: automatic 4 CTAs (s <= 8) or 8 (larger cells);
  // one CTA per cell with balancing or the translation step
  {
    int C = pin->cell_ctas == 0 ? (h->s <= 8 ? 4 : 8) : pin->cell_ctas;
    if (pin->balance || pin->cell_ti) C = 1;
    h->order_mode = pin->cell_ctas == 0 ? 0 : 1;
    const size_t rs = pin->precision ? sizeof(double) : sizeof(float);
    size_t smem = cell_smem_bytes(h->s, cap_side, cap_ny, pin->precision);
    int nctas = 0;
    for (; C > 1; C /= 2) {
      int cw = std::min(N, 256), ch = std::min(N, 128), nyl = 0;
      for (; cw >= 16; cw /= 2, ch = std::max(16, ch / 2)) {
        const size_t fixed = dist_smem_bytes(h->s, C, cw, ch, 0, pin->precision);
        if (fixed >= (size_t)smem_budget) continue;
        nyl = (int)(((size_t)smem_budget - fixed) / (5 * rs)) / 32 * 32;
        // epilogue scratch (3 nx1 W) must fit in the T/U/bl/lrho/Zv region
        if (nyl >= 512 && 4 * h->s * cw <= 2 * h->s * ch + 3 * nyl) break;
        nyl = 0;
      }
      if (nyl < 512) continue;
      const size_t sm = std::max(smem, dist_smem_bytes(h->s, C, cw, ch, nyl, pin->precision));
      const int n = cell_resident_ctas(sm, C, pin->precision);
      if (n >= C) {
        S.dist_c = C; S.dist_cap_w = cw; S.dist_cap_hl = ch; S.dist_cap_nyl = nyl;
        smem = sm;
        nctas = n;
        break;
      }
    }
    if (C <= 1) {
      S.dist_c = 1; S.dist_cap_w = S.dist_cap_hl = S.dist_cap_nyl = 0;
      h->order_mode = 2;
      nctas = cell_resident_ctas(smem, 1, pin->precision);
    }
    (void)nctas;
    h->cell_smem = smem;
    for (int k = 0, c = 1; k < 4; ++k, c *= 2)
      h->res[k] = c <= std::max(1, S.dist_c) ? cell_resident_ctas(smem, c, pin->precision) : 0;
    h->split = pin->cell_split > 0.0 ? pin->cell_split : 2.0;
    set_cluster(h, S.dist_c);
    if (S.dist_c > 1 &&
        (cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      h->st2 = nullptr;
    }
    set_cluster(h, S.dist_c);
  }
  std::vector<CellDesc> cells[2];
  for (int w = 0; w < 2; ++w) {
    build_partition(h, w, cells[w], h->sub_start[w]);
    h->ncell[w] = (int)cells[w].size();
  }
  int mb = 0;
  for (int w = 0; w < 2; ++w) {
    if (pin->strategy == DOMDEC_STAGGERED || pin->strategy == DOMDEC_STAGGERED_LINE) {
      for (int b = 0; b < 4; ++b) mb = std::max(mb, h->sub_start[w][b + 1] - h->sub_start[w][b]);
    } else {
      mb = std::max(mb, h->ncell[w]);
    }
  }
  h->max_batch = mb;
  cudaError_t e = cudaSuccess;
#define DD_ALLOC(ptr, cnt)                                  \
  do {                                                      \
    if ((e = dalloc(h, &(ptr), (cnt))) != cudaSuccess) {    \
      domdec_free(h);                                       \
      return DOMDEC_ENOMEM;                                 \
    }                                                       \
  } while (0)
  double *dmu, *dnu, *dlogmu, *dlognu, *dmuinu;
  DD_ALLOC(dmu, n); DD_ALLOC(dnu, n); DD_ALLOC(dlogmu, n); DD_ALLOC(dlognu, n);
  DD_ALLOC(S.alpha, n); DD_ALLOC(S.PX, n); DD_ALLOC(S.PY, n); DD_ALLOC(S.PXnew, n); DD_ALLOC(S.dPY, n); DD_ALLOC(S.alphanew, n);
  DD_ALLOC(S.Cc, h->nbasic); DD_ALLOC(S.Hh, h->nbasic); DD_ALLOC(dmuinu, h->nbasic);
  DD_ALLOC(h->d_mumass, h->nbasic);
  DD_ALLOC(S.box, h->nbasic);
  DD_ALLOC(S.cur, 1); DD_ALLOC(S.head, 1);
  DD_ALLOC(h->d_cells[0], std::max(1, h->ncell[0])); DD_ALLOC(h->d_cells[1], std::max(1, h->ncell[1]));
  DD_ALLOC(S.cout, std::max(1, mb));
  S.cap_nut = std::max(cap_ny, S.dist_c > 1 ? S.dist_c * S.dist_cap_nyl : 0);
  DD_ALLOC(S.nut, (size_t)std::max(1, mb) * 4 * S.cap_nut);
  DD_ALLOC(S.theta, 1); DD_ALLOC(S.declog, 4 * LOGCAP); DD_ALLOC(S.counters, NCOUNT);
  DD_ALLOC(S.slotctr, 1);
  DD_ALLOC(S.status, 1); DD_ALLOC(S.red, kRedBlocks * 5 + 8); DD_ALLOC(S.red_count, 1);
  DD_ALLOC(h->d_newoff, h->nbasic + 1); DD_ALLOC(h->d_scratch, 64);
  DD_ALLOC(h->d_partials, kRedBlocks * 8);
  DD_ALLOC(h->S.line, 16); DD_ALLOC(h->d_numom, 8);
  DD_ALLOC(S.queue, 2);
  DD_ALLOC(S.nbig, 8);
  DD_ALLOC(S.order[0], std::max(1, h->ncell[0])); DD_ALLOC(S.order[1], std::max(1, h->ncell[1]));
  {
    // spill slots for cell boxes beyond the shared-memory capacity: Y-side arrays
    // (4 s N + 5 N^2 values) followed by 4 N^2 doubles of new marginals
    const size_t rs = pin->precision ? sizeof(double) : sizeof(float);
    size_t ybytes = rs * (4 * (size_t)h->s * N + 5 * (size_t)n);
    ybytes = (ybytes + 255) / 256 * 256;
    const size_t stride = ybytes + 4 * (size_t)n * sizeof(double);
    // default: one slot per cell of the largest sub-batch, within 1 GiB
    const size_t budget = (size_t)1 << 30;
    int slots = (int)std::min<size_t>((size_t)std::max(1, mb), std::max<size_t>(1, budget / stride));
    if (pin->spill_slots > 0) slots = pin->spill_slots;
    if (pin->spill_slots < 0) slots = 0;
    S.spill_stride = (long long)stride;
    S.spill_nut_off = (long long)ybytes;
    S.spill_slots = slots;
    DD_ALLOC(S.spill, stride * std::max(slots, 1));
    DD_ALLOC(S.spill_count, 1);
  }
  S.mu = dmu; S.nu = dnu; S.logmu = dlogmu; S.lognu = dlognu; S.muinu = dmuinu;
  if (cudaMallocHost(&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) { domdec_free(h); return DOMDEC_ENOMEM; }
  cudaStream_t st = h->st;
  for (int w = 0; w < 2; ++w)
    if (h->ncell[w] &&
        cudaMemcpyAsync(h->d_cells[w], cells[w].data(), cells[w].size() * sizeof(CellDesc),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
      domdec_free(h);
      return DOMDEC_ECUDA;
    }
  for (int w = 0; w < 2; ++w) {
    S.cells[w] = h->d_cells[w];
    for (int b = 0; b < 5; ++b) S.sub_start[w][b] = h->sub_start[w][b];
  }
  S.staggered = pin->strategy == DOMDEC_STAGGERED || pin->strategy == DOMDEC_STAGGERED_LINE;
  S.newoff = h->d_newoff;
  h->eps0 = pin->eps;
  h->err0 = pin->err;
  rc = load_problem(h, mu, nu, alpha0, beta0, pin->eps_init);
  if (rc) {
    domdec_free(h);
    return rc;
  }
  *out = h;
  return DOMDEC_OK;
#undef DD_ALLOC
}

int domdec_iterate(domdec_t h, int n_sweeps) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (n_sweeps < 0) return DOMDEC_EINVAL;
  for (int k = 0; k < n_sweeps; ++k) {
    const int part = (int)(h->sweeps % 2);
    int rc = enqueue_sweep(h, part, h->slot);
    if (rc) return fail(h, rc);
    h->slot += batches_per_sweep(h, part);
    ++h->sweeps;
  }
  return DOMDEC_OK;
}

int domdec_autotune(domdec_t h, int* cluster_ctas, double* split_factor) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  struct Cand { int C; double f; };
  std::vector<Cand> cands = {{1, 2.0}};
  for (int k = 1, c = 2; k < 4; ++k, c *= 2) {
    if (c > h->S.dist_c || h->res[k] < c) continue;
    for (double f : {0.5, 1.0, 2.0}) cands.push_back({c, f});
  }
  double best = -1.0;
  Cand pick = {h->crun, h->split};
  cudaEvent_t e0 = take_event(h), e1 = take_event(h);
  for (const Cand& c : cands) {
    int rc = domdec_sync(h);
    if (rc < 0) return rc;
    unsigned long long it0 = 0, it1 = 0;
    if (cudaMemcpy(&it0, h->S.counters, sizeof(it0), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, DOMDEC_ECUDA);
    set_cluster(h, c.C);
    h->split = c.f;
    cudaEventRecord(e0, h->st);
    rc = domdec_iterate(h, 1);
    cudaEventRecord(e1, h->st);
    if (rc) return rc;
    rc = domdec_sync(h);
    if (rc < 0) return rc;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (cudaMemcpy(&it1, h->S.counters, sizeof(it1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(h, DOMDEC_ECUDA);
    const double rate = ms > 0.f ? (double)(it1 - it0) / ms : 0.0;
    if (h->crun == c.C && rate > best) { best = rate; pick = c; }
  }
  h->pool.push_back(e0);
  h->pool.push_back(e1);
  set_cluster(h, pick.C);
  h->split = pick.f;
  if (cluster_ctas) *cluster_ctas = h->crun;
  if (split_factor) *split_factor = h->split;
  return DOMDEC_OK;
}

int domdec_set_launch(domdec_t h, int cluster_ctas, double split_factor, int* effective_ctas) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if ((cluster_ctas != 1 && cluster_ctas != 2 && cluster_ctas != 4 && cluster_ctas != 8) ||
      !(split_factor > 0.0) || std::isinf(split_factor))
    return DOMDEC_EINVAL;
  set_cluster(h, cluster_ctas);
  h->split = split_factor;
  if (effective_ctas) *effective_ctas = h->crun;
  return DOMDEC_OK;
}

int domdec_reset(domdec_t h, const double* mu, const double* nu, const double* alpha0, const double* beta0,
                 double eps_init) {
  if (!h || !mu || !nu) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if ((alpha0 == nullptr) != (beta0 == nullptr)) return DOMDEC_EINVAL;
  if (alpha0 && !(eps_init > 0.0 && std::isfinite(eps_init))) return DOMDEC_EINVAL;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  prof_collect(h);
  h->S.eps = h->p.eps = h->eps0;
  h->S.err = h->p.err = h->err0;
  const int rc = load_problem(h, mu, nu, alpha0, beta0, eps_init);
  return rc ? fail(h, rc) : DOMDEC_OK;
}

int domdec_set_eps(domdec_t h, double eps) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (!(eps > 0.0) || !std::isfinite(eps)) return DOMDEC_EINVAL;
  h->S.eps = eps;
  h->p.eps = eps;
  return DOMDEC_OK;
}

int domdec_set_tolerance(domdec_t h, double err) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (!(err == err) || std::isinf(err)) return DOMDEC_EINVAL;
  h->S.err = err;
  h->p.err = err;
  return DOMDEC_OK;
}

int domdec_sync(domdec_t h) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  int rc = read_status(h);
  if (rc) return rc;
  rc = ensure_arena(h);
  if (rc) return rc;
  unsigned long long c[NCOUNT];
  if (cudaMemcpy(c, h->S.counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  // the warning covers the cell solves since the previous domdec_sync only
  const bool notconv = c[2] > h->maxit_seen;
  h->maxit_seen = c[2];
  return notconv ? DOMDEC_WNOTCONV : DOMDEC_OK;
}

int domdec_score(domdec_t h, double out[6]) {
  if (!h || !out) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (launch_score(h->S, h->d_scratch, h->st, h->d_partials) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  cudaMemcpyAsync(h->h_pinned, h->d_scratch, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  cudaMemcpyAsync(h->h_pinned + 8, h->S.theta, sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  int rc = read_status(h);
  if (rc) return rc;
  const double* v = h->h_pinned;
  out[0] = v[0] + v[1] + v[2];
  out[1] = v[0];
  out[2] = v[1];
  out[3] = v[2];
  out[4] = v[3];
  out[5] = h->h_pinned[8];
  return DOMDEC_OK;
}

int domdec_plan_marginals(domdec_t h, double* PX, double* PY) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  cudaError_t e = cudaSuccess;
  if (PX) e = cudaMemcpyAsync(PX, h->S.PX, h->n * sizeof(double), cudaMemcpyDefault, h->st);
  if (PY && e == cudaSuccess) e = cudaMemcpyAsync(PY, h->S.PY, h->n * sizeof(double), cudaMemcpyDefault, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  return read_status(h);
}

int domdec_duals(domdec_t h, double* alpha) {
  if (!h || !alpha) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  cudaError_t e = cudaMemcpyAsync(alpha, h->S.alpha, h->n * sizeof(double), cudaMemcpyDefault, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  return read_status(h);
}

int domdec_basic_costs(domdec_t h, double* C, double* H) {
  if (!h) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  cudaError_t e = cudaSuccess;
  if (C) e = cudaMemcpyAsync(C, h->S.Cc, h->nbasic * sizeof(double), cudaMemcpyDefault, h->st);
  if (H && e == cudaSuccess) e = cudaMemcpyAsync(H, h->S.Hh, h->nbasic * sizeof(double), cudaMemcpyDefault, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  return read_status(h);
}

int domdec_pd_gap(domdec_t h, double out[5], double* beta) {
  if (!h || !out) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  const int n = h->n;
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, 5 * (size_t)n * sizeof(double), h->st) != cudaSuccess) return fail(h, DOMDEC_ENOMEM);
  double *z = buf, *ba = buf + n, *bb = buf + 2 * (size_t)n, *bt = buf + 3 * (size_t)n, *bc = buf + 4 * (size_t)n;
  cudaError_t e = global_lse64(h->S.alpha, h->S.logmu, h->S.eps, h->S.h, h->N, z, ba, bb, bc, h->st);
  if (e == cudaSuccess) e = launch_cert(h->S, z, bt, h->d_scratch + 16, h->st, h->d_partials);
  if (e == cudaSuccess) e = launch_score(h->S, h->d_scratch, h->st, h->d_partials);
  if (e == cudaSuccess && beta) e = cudaMemcpyAsync(beta, bt, n * sizeof(double), cudaMemcpyDefault, h->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->h_pinned, h->d_scratch, 24 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  cudaFreeAsync(buf, h->st);
  if (e != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  int rc = read_status(h);
  if (rc) return rc;
  const double* v = h->h_pinned;
  const double* c = v + 16;
  const double eps = h->S.eps, lam = h->S.lam;
  const double P = v[0] + v[1] + v[2];
  const double D = eps * c[3] * c[4] - eps * c[0] - lam * c[1] - lam * c[2];
  out[0] = P;
  out[1] = D;
  out[2] = (P - D) / std::fabs(D);
  out[3] = c[5];
  out[4] = c[6];
  return DOMDEC_OK;
}

long long domdec_basic_marginals(domdec_t h, int* box, double* values, long long cap) {
  if (!h || !box) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  std::vector<BoxRec> b(h->nbasic);
  int cur = 0;
  if (cudaMemcpy(b.data(), h->S.box, h->nbasic * sizeof(BoxRec), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&cur, h->S.cur, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, DOMDEC_ECUDA);
  long long total = 0;
  for (int i = 0; i < h->nbasic; ++i) {
    box[4 * i] = b[i].k0; box[4 * i + 1] = b[i].l0; box[4 * i + 2] = b[i].H; box[4 * i + 3] = b[i].W;
    total += (long long)b[i].H * b[i].W;
  }
  if (!values) return total;
  if (total > cap) return DOMDEC_EINVAL;
  long long pos = 0;
  for (int i = 0; i < h->nbasic; ++i) {
    long long sz = (long long)b[i].H * b[i].W;
    if (sz && cudaMemcpy(values + pos, h->S.arena[cur] + b[i].off, sz * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
      return fail(h, DOMDEC_ECUDA);
    pos += sz;
  }
  return total;
}

int domdec_kernel_times(domdec_t h, double ms[4], long long launches[4], int reset) {
  if (!h || !ms || !launches) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  prof_collect(h);
  for (int k = 0; k < 4; ++k) {
    ms[k] = h->kt[k];
    launches[k] = h->kn[k];
    if (reset) { h->kt[k] = 0.0; h->kn[k] = 0; }
  }
  return read_status(h);
}

int domdec_decision_log(domdec_t h, double* out, int max_records) {
  if (!h || !out || max_records < 0) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  std::vector<double> all(4 * LOGCAP);
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(all.data(), h->S.declog, all.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, DOMDEC_ECUDA);
  const long long have = std::min<long long>(h->slot, LOGCAP);
  const int cnt = (int)std::min<long long>(have, max_records);
  for (int k = 0; k < cnt; ++k) {
    const long long rec = h->slot - cnt + k;
    for (int j = 0; j < 4; ++j) out[4 * k + j] = all[4 * (rec % LOGCAP) + j];
  }
  return cnt;
}

int domdec_cell_log(domdec_t h, double* out, int max_records) {
  if (!h || !out || max_records < 0) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  const int cnt = std::min(h->last_batch, max_records);
  std::vector<CellOut> rec(std::max(cnt, 1));
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      (cnt && cudaMemcpy(rec.data(), h->S.cout, cnt * sizeof(CellOut), cudaMemcpyDeviceToHost) != cudaSuccess))
    return fail(h, DOMDEC_ECUDA);
  for (int j = 0; j < cnt; ++j) {
    const CellOut& o = rec[j];
    double* r = out + 9 * j;
    r[0] = o.k0; r[1] = o.l0; r[2] = o.H; r[3] = o.W; r[4] = o.iters; r[5] = o.status; r[6] = o.gap; r[7] = o.slot;
    r[8] = o.usec;
  }
  return cnt;
}

int domdec_get_stats(domdec_t h, domdec_stats* s) {
  if (!h || !s) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  unsigned long long c[NCOUNT];
  if (launch_score(h->S, h->d_scratch, h->st, h->d_partials) != cudaSuccess) return fail(h, DOMDEC_ECUDA);
  cudaMemcpyAsync(h->h_pinned, h->d_scratch, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->st);
  if (cudaStreamSynchronize(h->st) != cudaSuccess ||
      cudaMemcpy(c, h->S.counters, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, DOMDEC_ECUDA);
  s->sweeps = h->sweeps;
  s->cell_iters = (long long)c[0];
  s->cell_solves = (long long)c[1];
  s->maxit_cells = (long long)c[2];
  s->greedy_steps = (long long)c[3];
  s->safe_steps = (long long)c[4];
  s->lse_terms = (long long)c[7];
  s->box_points = (long long)c[8];
  s->arena_regrows = h->arena_regrows;
  s->cluster_regroups = h->regroups;
  s->max_cell_iters = (int)c[5];
  s->max_ny = (int)c[6];
  s->box_entries = (long long)h->h_pinned[4];
  return read_status(h);
}

int domdec_full_sinkhorn(const double* mu, const double* nu, int N, double eps_start, double eps, double lambda,
                         int variant, int precision, int maxit, double err, int check_every,
                         const double* beta_in, double* alpha, double* beta, double out[4], void* stream) {
  if (!mu || !nu || !out || N <= 0) return DOMDEC_EINVAL;
  const int var = variant & ~DOMDEC_SINKHORN_TI;
  if (!(eps > 0.0) || !(lambda > 0.0) || (var != 0 && var != 1) || precision < 0 || precision > 2 || maxit < 1)
    return DOMDEC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = N * N;
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, (6 * (size_t)n + 8) * sizeof(double), st) != cudaSuccess) return DOMDEC_ENOMEM;
  double *dmu = buf, *dnu = buf + n, *lmu = buf + 2 * (size_t)n, *lnu = buf + 3 * (size_t)n;
  double *da = buf + 4 * (size_t)n, *db = buf + 5 * (size_t)n, *dev = buf + 6 * (size_t)n;
  int* dstatus = nullptr;
  cudaError_t e = cudaMallocAsync(&dstatus, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dstatus, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dmu, mu, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dnu, nu, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    if (beta_in) e = cudaMemcpyAsync(db, beta_in, n * sizeof(double), cudaMemcpyDefault, st);
    else e = cudaMemsetAsync(db, 0, n * sizeof(double), st);
  }
  if (e == cudaSuccess) e = launch_prepare_inputs(dmu, dnu, lmu, lnu, n, dstatus, st);
  int hstat = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int rc = DOMDEC_OK;
  if (e != cudaSuccess) rc = DOMDEC_ECUDA;
  else if (hstat) rc = DOMDEC_EINVAL;
  if (rc == DOMDEC_OK) {
    cudaError_t ce = cudaSuccess;
    int r = full_sinkhorn_dev(dmu, dnu, lmu, lnu, N, eps_start, eps, lambda, variant, precision, maxit, err,
                              check_every, da, db, out, dev, st, &ce);
    if (r < 0) rc = DOMDEC_ECUDA;
    else {
      rc = r ? DOMDEC_WNOTCONV : DOMDEC_OK;
      if (alpha) e = cudaMemcpyAsync(alpha, da, n * sizeof(double), cudaMemcpyDefault, st);
      if (beta && e == cudaSuccess) e = cudaMemcpyAsync(beta, db, n * sizeof(double), cudaMemcpyDefault, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = DOMDEC_ECUDA;
    }
  }
  cudaFreeAsync(dstatus, st);
  cudaFreeAsync(buf, st);
  cudaStreamSynchronize(st);
  return rc;
}


// ---------------------------------------------------------------- gradients
namespace {
// Runs the adjoint on device arrays and copies the results to the caller's
// buffers (host or device; each may be NULL).  Returns a DOMDEC_* code.
int gradients_run(const double* dmu, const double* dnu, const double* dalpha, const double* dbeta, int N,
                  double eps, double lam, int precision, double* grad_mu, double* grad_nu, double* grad_x,
                  double out[5], cudaStream_t st) {
  const size_t n = (size_t)N * N;
  const size_t sb = adjoint_scratch_size(N, precision);
  unsigned char* buf = nullptr;
  const size_t head = (4 * n + 8) * sizeof(double) + 256;  // gm, gn, gx (2n), out; then 256-aligned scratch
  if (cudaMallocAsync(&buf, head + sb, st) != cudaSuccess) return DOMDEC_ENOMEM;
  double* gm = reinterpret_cast<double*>(buf);
  double* gn = gm + n;
  double* gx = gn + n;           // 2 n
  double* dout = gx + 2 * n;     // 8
  int* dbad = reinterpret_cast<int*>(dout + 7);
  unsigned char* scratch =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dout + 8) + 255) & ~uintptr_t(255));
  cudaError_t e = cudaMemsetAsync(dbad, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = adjoint_dev(dmu, dnu, dalpha, dbeta, N, eps, lam, precision, gm, gn, gx, dout, scratch, dbad, st);
  double hout[8];
  if (e == cudaSuccess) e = cudaMemcpyAsync(hout, dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad_mu) e = cudaMemcpyAsync(grad_mu, gm, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess && grad_nu) e = cudaMemcpyAsync(grad_nu, gn, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess && grad_x) e = cudaMemcpyAsync(grad_x, gx, 2 * n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  int bad = 0;
  std::memcpy(&bad, &hout[7], sizeof(int));
  if (bad) return DOMDEC_EINVAL;
  if (out) for (int k = 0; k < 5; ++k) out[k] = hout[k];
  return DOMDEC_OK;
}
}  // namespace

int domdec_uot_gradients(const double* mu, const double* nu, const double* alpha, const double* beta, int N,
                         double eps, double lambda, int precision, double* grad_mu, double* grad_nu,
                         double* grad_x, double out[5], void* stream) {
  if (!mu || !nu || !alpha || !beta || N <= 0 || N > 4096) return DOMDEC_EINVAL;
  if (!(eps > 0.0) || !(lambda > 0.0) || (precision != DOMDEC_FP32 && precision != DOMDEC_FP64))
    return DOMDEC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = (size_t)N * N;
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, 4 * n * sizeof(double), st) != cudaSuccess) return DOMDEC_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(buf, mu, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + n, nu, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + 2 * n, alpha, n * sizeof(double), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(buf + 3 * n, beta, n * sizeof(double), cudaMemcpyDefault, st);
  int rc = e == cudaSuccess ? gradients_run(buf, buf + n, buf + 2 * n, buf + 3 * n, N, eps, lambda, precision,
                                            grad_mu, grad_nu, grad_x, out, st)
                            : DOMDEC_ECUDA;
  cudaFreeAsync(buf, st);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == DOMDEC_OK) rc = DOMDEC_ECUDA;
  return rc;
}

int domdec_gradients(domdec_t h, int precision, double* grad_mu, double* grad_nu, double* grad_x,
                     double out[5], double* beta) {
  if (!h) return DOMDEC_EINVAL;
  if (precision != DOMDEC_FP32 && precision != DOMDEC_FP64) return DOMDEC_EINVAL;
  if (h->sticky) return DOMDEC_ESTATE;
  if (h->N > 4096) return DOMDEC_EINVAL;
  const int n = h->n;
  double* buf = nullptr;
  if (cudaMallocAsync(&buf, 5 * (size_t)n * sizeof(double), h->st) != cudaSuccess) return fail(h, DOMDEC_ENOMEM);
  double *z = buf, *ba = buf + n, *bb = buf + 2 * (size_t)n, *bt = buf + 3 * (size_t)n, *bc = buf + 4 * (size_t)n;
  // beta_star: one global closed-form Y-half of the stitched alpha (Eq. sinkhorn-iters-ot)
  cudaError_t e = global_lse64(h->S.alpha, h->S.logmu, h->S.eps, h->S.h, h->N, z, ba, bb, bc, h->st);
  if (e == cudaSuccess) e = launch_cert(h->S, z, bt, h->d_scratch + 16, h->st, h->d_partials);
  if (e == cudaSuccess && beta) e = cudaMemcpyAsync(beta, bt, n * sizeof(double), cudaMemcpyDefault, h->st);
  int rc = e == cudaSuccess ? gradients_run(h->S.mu, h->S.nu, h->S.alpha, bt, h->N, h->S.eps, h->S.lam, precision,
                                            grad_mu, grad_nu, grad_x, out, h->st)
                            : DOMDEC_ECUDA;
  cudaFreeAsync(buf, h->st);
  if (cudaStreamSynchronize(h->st) != cudaSuccess) rc = DOMDEC_ECUDA;
  if (rc == DOMDEC_ECUDA || rc == DOMDEC_ENOMEM) return fail(h, rc);
  if (rc) return rc;
  return read_status(h);
}

// ---------------------------------------------------------------- batches
struct domdec_batch_s {
  std::vector<domdec_t> hs;
  cudaStream_t st = nullptr;
  DevState* d_states = nullptr;
  CellRef* d_refs = nullptr;           // all reference lists, back to back
  int ref_off[2][5] = {{0}};           // list (part, sub) starts at ref_off; sub 4 = whole partition
  int ref_cnt[2][5] = {{0}};
  unsigned int* d_queue = nullptr;     // two work counters of the cell kernel
  int* d_order = nullptr;              // reference order of a launch (k_ref_order)
  int* d_nbig = nullptr;
  int precision = 0, maxn = 0, max_nbasic = 0, max_ref = 0;
  size_t smem = 0;                     // dynamic shared memory of the cell kernel (largest of the handles')
  int c_max = 1;                       // largest cluster size every instance's layout allows
  int res[4] = {0, 0, 0, 0};           // resident CTAs with clusters of 1, 2, 4, 8
  int C = 0;                           // cluster size of the sweeps (0: automatic)
  double factor = 2.0;                 // cluster-split threshold in mean works per CTA
  long long sweeps = 0;
  std::vector<DevState> host_states;
};

int domdec_batch_create(domdec_batch_t* out, domdec_t* handles, int n) {
  if (!out || !handles || n < 1) return DOMDEC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return DOMDEC_EINVAL;
    if (handles[i]->sticky) return DOMDEC_ESTATE;
    if (handles[i]->p.precision != handles[0]->p.precision || handles[i]->p.strategy != handles[0]->p.strategy ||
        handles[i]->sweeps != handles[0]->sweeps || handles[i]->p.strategy == DOMDEC_LINE ||
        handles[i]->p.strategy == DOMDEC_STAGGERED_LINE ||
        handles[i]->p.balance)
      return DOMDEC_EINVAL;
  }
  domdec_batch_s* b = new (std::nothrow) domdec_batch_s();
  if (!b) return DOMDEC_ENOMEM;
  b->hs.assign(handles, handles + n);
  b->st = handles[0]->st;
  b->precision = handles[0]->p.precision;
  b->sweeps = handles[0]->sweeps;
  b->c_max = 8;
  for (auto h : b->hs) {
    b->smem = std::max(b->smem, h->cell_smem);
    b->c_max = std::min(b->c_max, std::max(1, h->S.dist_c));
    b->maxn = std::max(b->maxn, h->N);
    b->max_nbasic = std::max(b->max_nbasic, h->nbasic);
  }
  for (int k = 0, c = 1; k < 4; ++k, c *= 2)
    b->res[k] = c <= b->c_max ? cell_multi_resident_ctas(b->smem, c, b->precision) : 0;
  // reference lists: for each (partition, sub-batch) the cells of every
  // instance, larger grids first (their boxes are larger: longest jobs first)
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return handles[x]->N > handles[y]->N; });
  std::vector<CellRef> refs;
  for (int part = 0; part < 2; ++part)
    for (int sub = 0; sub < 5; ++sub) {
      b->ref_off[part][sub] = (int)refs.size();
      for (int i : order) {
        domdec_t h = handles[i];
        const int beg = sub < 4 ? h->sub_start[part][sub] : 0;
        const int end = sub < 4 ? h->sub_start[part][sub + 1] : h->ncell[part];
        for (int c = beg; c < end; ++c) refs.push_back({i, c, c - beg, end - beg});
      }
      b->ref_cnt[part][sub] = (int)refs.size() - b->ref_off[part][sub];
    }
  for (int part = 0; part < 2; ++part)
    for (int sub = 0; sub < 5; ++sub) b->max_ref = std::max(b->max_ref, b->ref_cnt[part][sub]);
  if (cudaMalloc(&b->d_states, n * sizeof(DevState)) != cudaSuccess ||
      cudaMalloc(&b->d_refs, std::max<size_t>(1, refs.size()) * sizeof(CellRef)) != cudaSuccess ||
      cudaMalloc(&b->d_queue, 2 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&b->d_order, std::max(1, b->max_ref) * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_nbig, sizeof(int)) != cudaSuccess) {
    domdec_batch_free(b);
    return DOMDEC_ENOMEM;
  }
  if (!refs.empty() &&
      cudaMemcpy(b->d_refs, refs.data(), refs.size() * sizeof(CellRef), cudaMemcpyHostToDevice) != cudaSuccess) {
    domdec_batch_free(b);
    return DOMDEC_ECUDA;
  }
  *out = b;
  return DOMDEC_OK;
}

void domdec_batch_free(domdec_batch_t b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->d_states) cudaFree(b->d_states);
  if (b->d_refs) cudaFree(b->d_refs);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_nbig) cudaFree(b->d_nbig);
  delete b;
}

static int batch_upload(domdec_batch_t b) {
  b->host_states.resize(b->hs.size());
  for (size_t i = 0; i < b->hs.size(); ++i) {
    if (b->hs[i]->sticky) return DOMDEC_ESTATE;
    b->host_states[i] = b->hs[i]->S;
  }
  if (cudaMemcpyAsync(b->d_states, b->host_states.data(), b->hs.size() * sizeof(DevState),
                      cudaMemcpyHostToDevice, b->st) != cudaSuccess)
    return DOMDEC_ECUDA;
  return DOMDEC_OK;
}

// One sweep of every instance with clusters of C CTAs (0: automatic) and the
// cluster-split threshold `factor`.
static int batch_enqueue_sweep(domdec_batch_t b, int C, double factor) {
  const int part = (int)(b->sweeps % 2);
  const int ninst = (int)b->hs.size();
  const bool stag = b->hs[0]->p.strategy == DOMDEC_STAGGERED;
  const int subs[4] = {0, 1, 2, 3};
  const int nsub = stag ? 4 : 1;
  if (C <= 0) C = b->c_max >= 4 ? 4 : b->c_max;
  int ci = 0;
  while ((1 << ci) < C) ++ci;
  if (ci > 3 || b->res[ci] < C) { C = 1; ci = 0; }
  const int nctas = std::max(C, b->res[ci]);
  for (int k = 0; k < nsub; ++k) {
    const int sub = stag ? subs[k] : 4;
    const int nref = b->ref_cnt[part][sub];
    if (nref == 0) continue;
    const CellRef* refs = b->d_refs + b->ref_off[part][sub];
    if (launch_cell_solve_multi(b->d_states, refs, nref, part, b->d_order, b->d_nbig, b->d_queue, b->smem,
                                b->precision, C, factor, nctas, b->st) != cudaSuccess)
      return DOMDEC_ECUDA;
  if (launch_decide_multi(b->d_states, ninst, b->maxn, part, stag ? sub : -1, b->st) != cudaSuccess)
      return DOMDEC_ECUDA;
    if (launch_apply_multi(b->d_states, refs, nref, part, b->st) != cudaSuccess) return DOMDEC_ECUDA;
  }
  if (launch_compact_multi(b->d_states, ninst, b->max_nbasic, b->st) != cudaSuccess) return DOMDEC_ECUDA;
  for (auto h : b->hs) {
    h->slot += batches_per_sweep(h, part);
    ++h->sweeps;
  }
  ++b->sweeps;
  return DOMDEC_OK;
}

int domdec_batch_iterate(domdec_batch_t b, int n_sweeps) {
  if (!b || n_sweeps < 0) return DOMDEC_EINVAL;
  int rc = batch_upload(b);
  if (rc) return rc;
  for (int k = 0; k < n_sweeps; ++k) {
    rc = batch_enqueue_sweep(b, b->C, b->factor);
    if (rc) {
      for (auto h : b->hs) fail(h, rc);
      return rc;
    }
  }
  return DOMDEC_OK;
}

int domdec_batch_sync(domdec_batch_t b) {
  if (!b) return DOMDEC_EINVAL;
  int worst = DOMDEC_OK;
  for (auto h : b->hs) {
    int rc = domdec_sync(h);
    if (rc < 0) return rc;
    if (rc > worst) worst = rc;
  }
  return worst;
}

int domdec_batch_autotune(domdec_batch_t b, int* cluster_ctas, double* split_factor) {
  if (!b) return DOMDEC_EINVAL;
  // candidates: one CTA per cell, or clusters of 2 / 4 CTAs for the cells above
  // 1, 2 or 4 mean works per CTA (and those too large for one CTA); one sweep
  // each, timed with CUDA events; the highest cell-iteration rate is kept
  struct Cand { int C; double f; };
  std::vector<Cand> cands = {{1, 2.0}};
  for (int C = 2; C <= std::min(4, b->c_max); C *= 2) {
    int ci = C == 2 ? 1 : 2;
    if (b->res[ci] < C) continue;
    for (double f : {1.0, 2.0, 4.0}) cands.push_back({C, f});
  }
  double best = -1.0;
  Cand pick = cands[0];
  for (const Cand& c : cands) {
    int rc = domdec_batch_sync(b);
    if (rc < 0) return rc;
    long long it0 = 0;
    for (auto h : b->hs) {
      domdec_stats st;
      if (domdec_get_stats(h, &st)) return DOMDEC_ECUDA;
      it0 += st.cell_iters;
    }
    rc = batch_upload(b);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, b->st);
    rc = batch_enqueue_sweep(b, c.C, c.f);
    cudaEventRecord(e1, b->st);
    if (rc) return rc;
    rc = domdec_batch_sync(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc < 0) return rc;
    long long it1 = 0;
    for (auto h : b->hs) {
      domdec_stats st;
      if (domdec_get_stats(h, &st)) return DOMDEC_ECUDA;
      it1 += st.cell_iters;
    }
    const double rate = ms > 0.f ? (double)(it1 - it0) / ms : 0.0;
    if (rate > best) { best = rate; pick = c; }
  }
  b->C = pick.C;
  b->factor = pick.f;
  if (cluster_ctas) *cluster_ctas = pick.C;
  if (split_factor) *split_factor = pick.f;
  return DOMDEC_OK;
}
}  // extern "C"
