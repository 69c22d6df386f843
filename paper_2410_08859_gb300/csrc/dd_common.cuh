// Shared device definitions of the domain-decomposition library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dd_log_table.cuh"

#define DD_LOG2E 1.4426950408889634
#define DD_LN2 0.6931471805599453

// ---------------------------------------------------------------- status codes
// Per-cell status written by the cell kernel (CELL_SKIPPED: the launch found
// the handle halted and solved nothing).
enum { CELL_OK = 0, CELL_MAXIT = 1, CELL_EMPTY = 2, CELL_TOOBIG = 3, CELL_NONFINITE = 4, CELL_SKIPPED = 5 };
// Bits of the handle's device status word.  Two of them halt the enqueued
// sweeps (ST_HALT): every later sweep kernel leaves the state untouched until
// the host has handled the cause and re-enqueued the sub-batches that did not
// run.  ST_ARENA: a sub-batch's new boxes would not fit the arena (set by the
// decision kernel before any state changed; the host grows the arena).
// ST_REGROUP: a cell fits neither one CTA nor a cluster of the launch's size
// but does fit the layout's largest cluster (set by the ordering kernel before
// the sub-batch's cell solve; the host switches to that cluster size).
// ST_ARENA_LOST: the allocation guard of the mixing kernel fired (state lost).
enum { ST_TOOBIG = 1, ST_ARENA = 2, ST_EMPTY = 4, ST_NONFINITE = 8, ST_BADINPUT = 16, ST_ARENA_LOST = 32,
       ST_REGROUP = 64, ST_HALT = ST_ARENA | ST_REGROUP };

// ------------------------------------------------------------------ geometry
// One composite cell: its X box [i0, i0+nx1) x [j0, j0+nx2) (always a
// rectangle of real pixels, also for the clipped boundary cells of partition
// B) and the basic cell of each quadrant (row half, column half) relative to
// the X box origin; -1 where the quadrant does not exist.
struct CellDesc {
  int i0, j0, nx1, nx2;
  int mem[4];
};

// Output record of one cell solve.
struct CellOut {
  int k0, l0, H, W;      // the cell's Y box B_J
  int iters, status, D1, D2;
  int slot, usec;        // spill slot of an oversized box (-1: none); duration of the solve (microseconds)
  double Ct[4], Ht[4], mass[4];  // per quadrant: <c, pi~_i>, KL(pi~_i | mu_i x nu), |nu~_i|
  double dKX[2];         // sum_{x in X_J} [mu phi(P'/mu) - mu phi(P/mu)] for theta = 1 and theta_safe
  double gap;            // last PD/lam of the cell
};

// Basic-cell box: Y rows [k0, k0+H), columns [l0, l0+W), values at arena[off..].
struct BoxRec {
  int k0, l0, H, W;
  long long off;
};

// Everything the sweep kernels need; passed by value.
struct DevState {
  int N, s, nb, nbasic;
  double h, eps, lam, thr, err, tau;
  int maxit, newton_maxit, strategy, margin;
  int ti;                       // translation step after each cell X-half (0/1)
  double* line;                 // GetWeights_line state (16 doubles)
  int balance;                  // balancing step after each cell solve (0/1; one CTA per cell)
  int cap_ny, cap_side;
  int cap_nut;                  // new marginals per quadrant in a cell position's buffer (>= cap_ny, and the
                                //   cluster capacity dist_c * dist_cap_nyl)
  unsigned char* spill;         // spill slots: Y-side arrays and new marginals of cells too large
  long long spill_stride;       //   for shared memory (bytes per slot)
  long long spill_nut_off;      //   byte offset of the new marginals (4 N^2 doubles) inside a slot
  int spill_slots;              //   number of slots
  unsigned int* spill_count;    //   slots taken in the current launch (reset by k_decide)
  const double *mu, *nu, *logmu, *lognu;
  double* muinu;                // muinu[i] = |mu_i| |nu|
  double *alpha, *PX, *PY, *PXnew, *dPY;
  double* alphanew;             // the cell solves' new alpha on X_J, committed by the mixing kernel
                                // (so a halted sub-batch is solved again from the same alpha)
  double *Cc, *Hh;
  BoxRec* box;
  double* arena[2];
  int* cur;                     // index of the live arena
  unsigned long long* head;     // bump allocator of the live arena
  long long cap;                // capacity of each arena (doubles)
  CellOut* cout;
  double* nut;                  // per cell position: 4 * cap_nut new marginals
  double* theta;                // device scalar: last theta
  double* declog;               // per sub-batch: E0, E(1), E(safe), theta
  unsigned long long* counters; // 0 cell_iters, 1 cell_solves, 2 maxit cells, 3 greedy, 4 safe, 5 max iters,
                                // 6 max ny, 7 lse terms, 8 Y-box points of the cell solves
  int* status;
  double* red;                  // reduction scratch
  unsigned int* red_count;
  // partitions (for kernels that locate their own sub-batch)
  const CellDesc* cells[2];     // cells of partitions A and B, sorted by sub-batch
  int sub_start[2][5];          // sub-batch b of partition p: cells [sub_start[p][b], sub_start[p][b+1])
  int staggered;                // 1: four sub-batches per sweep, 0: one batch of all cells
  unsigned long long* slotctr;  // decision-log records written so far
  long long* newoff;            // compaction scratch: nbasic + 1 offsets
  unsigned int* queue;          // work queues of the persistent cell kernel: [0] cluster phase,
                                //   [1] single-CTA phase (reset by k_decide)
  int* order[2];                // per partition: cells of each sub-batch, cluster cells first, each
                                //   group by decreasing estimated work (k_cell_order)
  int* nbig;                    // [part * 4 + sub]: leading cells of the order solved by a whole cluster
  // capacities of the cluster-distributed cell solve (one cell over dist_c CTAs, split by Y rows)
  int dist_c;                   // CTAs per cluster (1: no cluster phase)
  int dist_cap_w;               // largest Y-box width
  int dist_cap_hl;              // largest number of Y rows per CTA
  int dist_cap_nyl;             // largest number of Y points per CTA
};

#define DD_LOGCAP 4096          // decision-log records kept per instance

// One cell of a many-instance launch: instance, cell index in its partition
// list, and its position within the instance's sub-batch.
struct CellRef {
  int inst, cell, pos, nbatch;
};

// Global nanosecond timer (the same on every SM).
__device__ __forceinline__ unsigned long long dd_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------------ math
__device__ __forceinline__ float dd_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float dd_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float dd_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double dd_ex2(double x) { return exp2(x); }
__device__ __forceinline__ double dd_lg2(double x) { return log2(x); }
__device__ __forceinline__ double dd_rcp(double x) { return 1.0 / x; }

template <typename R> __device__ __forceinline__ R dd_inf() { return R(INFINITY); }

// psi(d) = d e^d - e^d + 1 = e^{-g} KL-term ratio (phi(e^d) with phi(s) = s log s - s + 1),
// evaluated by its Taylor series sum_{k>=2} (k-1)/k! d^k near 0 to avoid cancellation.
template <typename R> __device__ __forceinline__ R dd_psi(R d) {
  const R lim = sizeof(R) == 4 ? R(0.25) : R(0.05);
  if (fabs(d) < lim) {
    R d2 = d * d;
    R poly = R(1.0 / 2) + d * (R(1.0 / 3) + d * (R(1.0 / 8) + d * (R(1.0 / 30) + d * (R(1.0 / 144)
             + d * (R(1.0 / 840) + d * (R(1.0 / 5760) + d * (R(1.0 / 45360) + d * R(1.0 / 403200))))))));
    return d2 * poly;
  }
  R e = dd_ex2(d * R(DD_LOG2E));
  return e * (d - R(1)) + R(1);
}

// Natural logarithm of a positive finite double by Tang's table-driven method
// (ACM TOMS 16, 1990): x = 2^e m with m in [0.75, 1.5) (so e = 0 on all of
// [0.75, 1.5) and no cancellation between e log 2 and log c near x = 1);
// c_j = 1 + j/128 is the nearest to m (j = -32..64); f = m - c_j is exact;
// r = f / c_j as f times the rounded reciprocal (|r| <= 2^-7.6); log1p(r) by
// its Taylor polynomial up to r^7 (remainder below 2^-56 relative);
// log x = e log 2 + log c_j + log1p(r).  About 12 FP64 operations against the
// library logarithm's longer sequence; the GPU test compares it with CUDA's
// log (a few ulp).  The tables are generated by gen_log_table.py.
__device__ __forceinline__ double dd_log(double x) {
  int hi = __double2hiint(x);
  int lo = __double2loint(x);
  int e = 0;
  if (hi < 0x00100000) {   // subnormal: scale into the normal range
    x *= 18014398509481984.0;   // 2^54
    hi = __double2hiint(x);
    lo = __double2loint(x);
    e = -54;
  }
  e += (hi >> 20) - 1023;
  double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // [1, 2)
  if (m >= 1.5) {
    m *= 0.5;
    e += 1;
  }
  const int j = __double2int_rn((m - 1.0) * 128.0);   // -32..64; m - 1 is exact
  const double f = m - (1.0 + j * 0.0078125);
  const double r = f * kInvC[j + 32];
  double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  p = fma(p, r, 0.2);
  p = fma(p, r, -0.25);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  const double l1p = fma(p, r * r, r);
  return fma((double)e, 0.6931471805599453, kLogC[j + 32] + l1p);
}

// mu phi(p/mu) with phi(s) = s log s - s + 1 (phi(0) = 1), in double.
__device__ __forceinline__ double dd_kl_term(double p, double m) {
  if (p <= 0.0) return m;
  return p * log(p / m) - p + m;
}

// ------------------------------------------------------------- reductions
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of K values per thread; result valid in every thread.
// Warp 0 adds the per-warp partials in a fixed order (deterministic).
// `scratch` must hold 32*K values of type T; ends with a barrier.
template <int K, typename T>
__device__ __forceinline__ void block_sum(T (&v)[K], T* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[wid * K + k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T a = lane < nw ? scratch[lane * K + k] : T(0);
      // fixed-order pairwise combination across the lanes
      a = warp_sum(a);
      if (lane == 0) scratch[32 * K + k] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = scratch[32 * K + k];
  __syncthreads();
}

// Two-stage grid reduction (deterministic): each of G blocks writes its K
// block sums to partials[blockIdx.x * K + k]; k_sum_partials then adds the G
// rows in block order.  With G = 1 the single block writes the result itself.
// G is at most kRedBlocks, a fixed grid (two blocks per SM of GB300's 152 SMs)
// that sizes the partial buffers; it is not a device query and any SM count works.
constexpr int kRedBlocks = 304;
inline int red_blocks(long long n, int threads, const double* partials) {
  if (!partials) return 1;
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > kRedBlocks ? kRedBlocks : g));
}
template <int K>
__device__ __forceinline__ void block_sum_to(double (&v)[K], double* scratch, double* dst) {
  block_sum<K>(v, scratch);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) dst[blockIdx.x * K + k] = v[k];
}
__global__ void k_sum_partials(const double* partials, int G, int K, double* out);

// New marginals of cell position j of the current launch (quadrant stride in *stride).
__device__ __forceinline__ double* cell_nut(const DevState& S, const CellOut& o, int j, int* stride) {
  if (o.slot >= 0) {
    *stride = S.N * S.N;
    return reinterpret_cast<double*>(S.spill + (long long)o.slot * S.spill_stride + S.spill_nut_off);
  }
  *stride = S.cap_nut;
  return S.nut + (long long)j * 4 * S.cap_nut;
}
