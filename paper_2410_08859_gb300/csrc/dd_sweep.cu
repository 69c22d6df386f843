// Sweep kernels other than the cell solve:
//  k_decide  -- GetWeights (greedy / safe / swift) for one sub-batch from FP64 score deltas (a6)
//  k_apply   -- pi' = sum_J (1-theta) pi_J + theta pi~_J on the basic-cell boxes, truncation,
//               tight boxes, P_Y / P_X / C_i / H_i updates (a7)
//  compaction of the box arena, initial plans, score and certificate reductions.
#include "dd_common.cuh"

// ============================================================== decision (a6)
// mu phi(p/mu) in float (the current score's marginal terms; see k_decide).
__device__ __forceinline__ float kl_term_f(double p, double m) {
  if (p <= 0.0) return (float)m;
  float pf = (float)p, mf = (float)m;
  return pf * (dd_lg2(pf / mf) * (float)DD_LN2) - pf + mf;
}

// mu phi(p/mu) in double from log mu (no division).
__device__ __forceinline__ double kl_term_log(double p, double m, double log_m) {
  if (p <= 0.0) return m;
  return p * (dd_log(p) - log_m) - p + m;
}

// Tracked score (the sum of per-basic-cell transport cost and entropy plus the
// two exact marginal penalties) and its value after mixing with theta = 1 and
// theta = 1/|b|; decision on the device, deterministic fixed-order reductions.
__device__ __forceinline__ void decide_body(const DevState& S, const CellDesc* __restrict__ cells, int begin,
                                            int nbatch, int bid, int nblk) {
  __shared__ double red[33 * 5];
  __shared__ bool is_last;
  __shared__ unsigned long long smax[2];   // largest iteration count and Y box of the sub-batch
  if (*(volatile int*)S.status & ST_HALT) return;   // halted until the host reruns the sub-batch
  if (threadIdx.x == 0) smax[0] = smax[1] = 0ull;
  const int n = S.N * S.N;
  const double lam = S.lam, eps = S.eps, th_s = 1.0 / nbatch;
  double v[5] = {0, 0, 0, 0, 0};
  // Every term that changes with the step is summed in double: on the pixels
  // where the sub-batch changes P_Y (dP_Y != 0) kl(p), kl(p + d) and
  // kl(p + d/|b|) all take double logarithms, so E(1) - E (the leniency test)
  // and E(1) - E(1/|b|) (the swift comparison) are exact to double rounding.
  // The terms that do not change (KL_X, and KL_Y where dP_Y = 0) cancel in both
  // differences and only set the scale E of the tie slack 1e-12 |E| and of the
  // leniency tau E (and the logged E): they are summed with float logarithms
  // (relative error ~1e-7 of E).
  for (int y = bid * blockDim.x + threadIdx.x; y < n; y += nblk * blockDim.x) {
    v[0] += (double)kl_term_f(S.PX[y], S.mu[y]);
    const double p = S.PY[y], d = S.dPY[y];
    if (d != 0.0) {
      const double m = S.nu[y], lm = S.lognu[y];
      const double k0 = kl_term_log(p, m, lm);
      const double k1 = kl_term_log(fmax(0.0, p + d), m, lm);
      v[1] += k0;
      v[2] += k1 - k0;
      v[3] += k1 - kl_term_log(fmax(0.0, p + th_s * d), m, lm);
    } else {
      v[1] += (double)kl_term_f(p, S.nu[y]);
    }
  }
  for (int i = bid * blockDim.x + threadIdx.x; i < S.nbasic; i += nblk * blockDim.x)
    v[4] += S.Cc[i] + eps * S.Hh[i];
  block_sum<5>(v, red);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) S.red[bid * 5 + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(S.red_count, 1u);
    is_last = (t == (unsigned int)nblk - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // last block: fixed-order reduction of the block partials and the per-cell terms
  // tot[9..13]: the sub-batch's cell-solve counters (iterations, solves, solves
  // stopped at maxit, exp terms, Y-box points), added to the handle's counters
  // only when the sub-batch goes ahead (a halted one is solved again later)
  double tot[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
    for (int k = 0; k < 5; ++k) tot[k] += ((volatile double*)S.red)[b * 5 + k];
  for (int j = threadIdx.x; j < nbatch; j += blockDim.x) {
    const CellOut& o = S.cout[j];
    if (o.status == CELL_EMPTY || o.status == CELL_TOOBIG) continue;
    const CellDesc cd = cells[begin + j];
    for (int q = 0; q < 4; ++q) {
      int bi = cd.mem[q];
      if (bi < 0) continue;
      tot[5] += (o.Ct[q] - S.Cc[bi]) + eps * (o.Ht[q] - S.Hh[bi]);
      tot[8] += (double)o.H * o.W;   // the new box of member q lies inside B_J
    }
    tot[6] += o.dKX[0];
    tot[7] += o.dKX[1];
    const double it = (double)o.iters, ny = (double)o.H * o.W;
    const double nx1 = cd.nx1, nx2 = cd.nx2;
    tot[9] += it;
    tot[10] += 1.0;
    tot[11] += o.status == CELL_MAXIT ? 1.0 : 0.0;
    // exp terms of one iteration: the two separable passes of each half
    tot[12] += it * (nx1 * nx2 * o.W + ny * nx1 + nx2 * ny + nx1 * nx2 * o.H);
    tot[13] += ny;
    atomicMax(&smax[0], (unsigned long long)o.iters);
    atomicMax(&smax[1], (unsigned long long)(o.H * o.W));
  }
  __shared__ double red14[33 * 14];
  block_sum<14>(tot, red14);
  if (threadIdx.x != 0) return;
  // reserve the arena space of the sub-batch's new boxes before anything changes
  if ((double)*S.head + tot[8] > (double)S.cap) {
    atomicOr(S.status, ST_ARENA);
    *S.red_count = 0u;
    if (S.spill_count) *S.spill_count = 0u;
    if (S.queue) { S.queue[0] = 0u; S.queue[1] = 0u; }
    return;
  }
  atomicAdd(S.counters + 0, (unsigned long long)tot[9]);
  atomicAdd(S.counters + 1, (unsigned long long)tot[10]);
  atomicAdd(S.counters + 2, (unsigned long long)tot[11]);
  atomicAdd(S.counters + 7, (unsigned long long)tot[12]);
  atomicAdd(S.counters + 8, (unsigned long long)tot[13]);
  atomicMax(S.counters + 5, smax[0]);
  atomicMax(S.counters + 6, smax[1]);
  const double dL = tot[5], dKX1 = tot[6], dKXs = tot[7];
  const double E0 = tot[4] + lam * tot[0] + lam * tot[1];
  const double dg = dL + lam * dKX1 + lam * tot[2];          // E(1) - E
  // E(1) - E(1/|b|) in double: the P_Y part directly, the rest as before
  const double dgs = (1.0 - th_s) * dL + lam * (dKX1 - dKXs) + lam * tot[3];
  const double ds = dg - dgs;                                // E(1/|b|) - E
  const double Eg = E0 + dg, Es = E0 + ds;
  double theta;
  if (S.strategy == 3) theta = 1.0;                 // greedy
  else if (S.strategy == 2) theta = th_s;           // safe
  else theta = (dgs <= 1e-12 * fabs(E0) || (S.tau > 0.0 && dg <= S.tau * E0)) ? 1.0 : th_s;
  *S.theta = theta;
  const unsigned long long slot = (*S.slotctr)++ % DD_LOGCAP;
  double* lg = S.declog + 4 * slot;
  lg[0] = E0; lg[1] = Eg; lg[2] = Es; lg[3] = theta;
  if (S.strategy == 4 || S.strategy == 5) {
    // GetWeights_line: the search kernels refine theta (and the log record)
    S.line[5] = 0.0;        // not done
    S.line[6] = th_s;       // lower end of the bracket
    S.line[7] = dL;         // linear part of E'(zeta)
  } else {
    atomicAdd(S.counters + (theta == 1.0 ? 3 : 4), 1ull);
  }
  *S.red_count = 0u;
  if (S.spill_count) *S.spill_count = 0u;
  if (S.queue) { S.queue[0] = 0u; S.queue[1] = 0u; }
}

__global__ void __launch_bounds__(512)
k_decide(DevState S, const CellDesc* __restrict__ cells, int begin, int nbatch) {
  decide_body(S, cells, begin, nbatch, blockIdx.x, gridDim.x);
}

// Many instances: blockIdx.y selects the instance; sub < 0 means the whole
// partition (non-staggered strategies).
__global__ void __launch_bounds__(512)
k_decide_multi(const DevState* __restrict__ states, int part, int sub) {
  __shared__ DevState sS;
  {
    const int* src = reinterpret_cast<const int*>(states + blockIdx.y);
    int* dst = reinterpret_cast<int*>(&sS);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const int begin = sub < 0 ? 0 : sS.sub_start[part][sub];
  const int end = sub < 0 ? sS.sub_start[part][4] : sS.sub_start[part][sub + 1];
  if (end <= begin) return;
  const int n = sS.N * sS.N;
  int nblk = (n + 511) / 512;
  if (nblk > (int)gridDim.x) nblk = gridDim.x;
  if ((int)blockIdx.x >= nblk) return;
  decide_body(sS, sS.cells[part], begin, end - begin, blockIdx.x, nblk);
}

// ====================================================== GetWeights_line (a6)
// E_hat(zeta) of sum_J (1-zeta) pi_J + zeta pi~_J is convex in zeta: C and H
// mix linearly, and so do the marginals inside the two KL terms.  With the
// marginal changes dX = P_X pi~ - P_X pi on the batch's X boxes and dY = dP_Y:
//   E'(zeta)  = L + lam <dX, log(P_X(zeta)/mu)> + lam <dY, log(P_Y(zeta)/nu)>
//   E''(zeta) = lam <dX^2, 1/P_X(zeta)> + lam <dY^2, 1/P_Y(zeta)>
// The minimiser on [lo, 1] (lo = 1/|b|) is 1 if E'(1) <= 0, lo if E'(lo) >= 0,
// else the root of E': Newton steps from zeta = 1 inside the bracket, the
// bracket's midpoint when a step leaves it or when the bracket has not halved
// over the last two steps; stop when |E'| <= 1e-12 x (sum of the magnitudes
// of its terms), when the bracket is narrower than 1e-12, or after 48 steps.
// State S.line: [0] a, [1] b, [2] zeta to evaluate, [3] g, [4] h, [5] done,
// [6] lo, [7] L, [8] width one step ago, [9] width two steps ago,
// [12..15] the summed terms of the last evaluation.
constexpr int kLineIters = 48;
constexpr double kLineGtol = 1e-12, kLineXtol = 1e-12, kLinePfloor = 1e-300;

// Block partials of [<d, log(p(z)/m)>, <d^2, 1/p(z)>, <|d log(p(z)/m)|>, <d, log(p(lo)/m)>]
// at z = 1 (first == 1, also at lo) or at z = S.line[2].
__global__ void __launch_bounds__(512)
k_line_eval(DevState S, const CellDesc* __restrict__ cells, int begin, int nbatch, int first, double* partials) {
  __shared__ double red[33 * 4];
  if (S.line[5] != 0.0 || (*(volatile int*)S.status & ST_HALT)) return;   // uniform across blocks
  const double z = first ? 1.0 : S.line[2], lo = S.line[6];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  auto term = [&](double p0, double d, double m) {
    const double p = fmax(p0 + z * d, kLinePfloor);
    const double t = d * log(p / m);
    v[0] += t;
    v[1] += d * d / p;
    v[2] += fabs(t);
    if (first) v[3] += d * log(fmax(p0 + lo * d, kLinePfloor) / m);
  };
  const int N = S.N;
  for (int j = blockIdx.x; j < nbatch; j += gridDim.x) {
    const CellOut& o = S.cout[j];
    if (o.status == CELL_EMPTY || o.status == CELL_TOOBIG) continue;
    const CellDesc cd = cells[begin + j];
    const int nx = cd.nx1 * cd.nx2;
    for (int t = threadIdx.x; t < nx; t += blockDim.x) {
      const int r = t / cd.nx2, c = t - r * cd.nx2;
      const int x = (cd.i0 + r) * N + cd.j0 + c;
      const double p0 = S.PX[x], d = S.PXnew[x] - p0;
      if (d != 0.0) term(p0, d, S.mu[x]);
    }
  }
  const int n = N * N;
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
    const double d = S.dPY[y];
    if (d != 0.0) term(S.PY[y], d, S.nu[y]);
  }
  block_sum_to<4>(v, red, partials);
}

// One step of the search from the sums of the last evaluation (one thread).
__global__ void k_line_step(DevState S, int first, int last) {
  if (threadIdx.x != 0 || S.line[5] != 0.0 || (*(volatile int*)S.status & ST_HALT)) return;
  double* L = S.line;
  const double lam = S.lam;
  const double g = L[7] + lam * L[12], h = lam * L[13], scale = fabs(L[7]) + lam * L[14];
  double a = L[0], b = L[1], z = first ? 1.0 : L[2];
  bool done = false;
  double zeta = z;
  if (first) {
    if (g <= 0.0) { done = true; zeta = 1.0; }
    else if (L[7] + lam * L[15] >= 0.0) { done = true; zeta = L[6]; }
    else { a = L[6]; b = 1.0; L[8] = INFINITY; L[9] = INFINITY; }
  } else {
    if (g > 0.0) b = z; else a = z;
    L[9] = L[8];
    L[8] = b - a;
    if (fabs(g) <= kLineGtol * scale || b - a <= kLineXtol || last) { done = true; zeta = z; }
  }
  if (!done) {
    double zn = h > 0.0 ? z - g / h : a;
    if (!(a < zn && zn < b) || (b - a) > 0.5 * L[9]) zn = 0.5 * (a + b);
    L[0] = a; L[1] = b; L[2] = zn; L[3] = g; L[4] = h;
    return;
  }
  L[5] = 1.0;
  *S.theta = zeta;
  const unsigned long long slot = (*S.slotctr + DD_LOGCAP - 1) % DD_LOGCAP;
  S.declog[4 * slot + 3] = zeta;
  atomicAdd(S.counters + (zeta == 1.0 ? 3 : 4), 1ull);
}

// ================================================================= apply (a7)
// One quadrant q (member basic cell cd.mem[q]) of cell position `pos`; the four
// quadrants of a cell run in four CTAs (the largest cell's work is split four ways).
__device__ __forceinline__ void apply_body(const DevState& S, const CellDesc cd, int pos, int q) {
  __shared__ BoxRec ob;
  __shared__ int bb[4];          // min kk, max kk, min ll, max ll of kept entries
  __shared__ long long noff;
  __shared__ int nbox[4];
  const CellOut o = S.cout[pos];
  if (o.status == CELL_EMPTY || o.status == CELL_TOOBIG || o.status == CELL_SKIPPED) return;
  const int N = S.N, H = o.H, W = o.W, ny = H * W;
  const int tid = threadIdx.x;
  // dP_Y of the sub-batch back to zero on this cell's box (each quadrant CTA a quarter)
  for (int u = 4 * tid + q; u < ny; u += 4 * blockDim.x) {
    int kk = u / W, ll = u - kk * W;
    S.dPY[(o.k0 + kk) * N + o.l0 + ll] = 0.0;
  }
  const int bi = cd.mem[q];
  if (bi < 0 || (*(volatile int*)S.status & ST_HALT)) return;
  const double th = *S.theta, thr = S.thr;
  double* arena = S.arena[*S.cur];
  int nst;
  // the new marginal of this quadrant; the first pass overwrites it with the mixed
  // value (nothing reads it after this kernel), which the second pass copies
  double* nut = cell_nut(S, o, pos, &nst);
  nut += (long long)q * nst;
  if (tid == 0) {
    ob = S.box[bi];
    bb[0] = 1 << 30; bb[1] = -1; bb[2] = 1 << 30; bb[3] = -1;
  }
  __syncthreads();
  int lb0 = 1 << 30, lb1 = -1, lb2 = 1 << 30, lb3 = -1;
  const BoxRec b = ob;
  for (int u = tid; u < ny; u += blockDim.x) {
    int kk = u / W, ll = u - kk * W;
    int y1 = o.k0 + kk, y2 = o.l0 + ll;
    int a = y1 - b.k0, c = y2 - b.l0;
    double old = (a >= 0 && c >= 0 && a < b.H && c < b.W) ? arena[b.off + (long long)a * b.W + c] : 0.0;
    double v = (1.0 - th) * old + th * nut[u];
    if (v < thr) v = 0.0;
    nut[u] = v;
    const double dl = v - old;
    if (v > 0.0) {
      lb0 = min(lb0, kk); lb1 = max(lb1, kk);
      lb2 = min(lb2, ll); lb3 = max(lb3, ll);
    }
    if (dl != 0.0) atomicAdd(S.PY + y1 * N + y2, dl);
  }
  {
    int m0 = warp_min(lb0), m1 = warp_max(lb1), m2 = warp_min(lb2), m3 = warp_max(lb3);
    if ((tid & 31) == 0) {
      atomicMin(&bb[0], m0); atomicMax(&bb[1], m1);
      atomicMin(&bb[2], m2); atomicMax(&bb[3], m3);
    }
  }
  __syncthreads();
  if (tid == 0) {
    BoxRec nb = {o.k0, o.l0, 0, 0, 0};
    if (bb[1] >= 0) {
      nb.k0 = o.k0 + bb[0]; nb.l0 = o.l0 + bb[2];
      nb.H = bb[1] - bb[0] + 1; nb.W = bb[3] - bb[2] + 1;
    }
    long long sz = (long long)nb.H * nb.W;
    unsigned long long off = atomicAdd(S.head, (unsigned long long)sz);
    if ((long long)off + sz > S.cap) {   // excluded by the reservation in k_decide
      atomicOr(S.status, ST_ARENA_LOST);
      nb.H = nb.W = 0;
      off = 0;
    }
    nb.off = (long long)off;
    noff = nb.off;
    nbox[0] = nb.k0; nbox[1] = nb.l0; nbox[2] = nb.H; nbox[3] = nb.W;
    S.box[bi] = nb;
    S.Cc[bi] = (1.0 - th) * S.Cc[bi] + th * o.Ct[q];
    S.Hh[bi] = (1.0 - th) * S.Hh[bi] + th * o.Ht[q];
  }
  __syncthreads();
  {
    const int nk0 = nbox[0], nl0 = nbox[1], nH = nbox[2], nW = nbox[3];
    for (int u = tid; u < nH * nW; u += blockDim.x) {
      int a = u / nW, c = u - a * nW;
      const int y1 = nk0 + a, y2 = nl0 + c;
      arena[noff + u] = nut[(y1 - o.k0) * W + (y2 - o.l0)];
    }
  }
  // P_X on the quadrant's pixels, and the cell's new alpha there
  const int s = S.s, hr = q >> 1, hc = q & 1;
  const int rb = hr * s, re = min(cd.nx1, rb + s), cb = hc * s, ce = min(cd.nx2, cb + s);
  const int qw = ce - cb;
  for (int t = tid; t < (re - rb) * qw; t += blockDim.x) {
    int r = rb + t / qw, c = cb + (t - (t / qw) * qw);
    int x = (cd.i0 + r) * N + cd.j0 + c;
    S.PX[x] = (1.0 - th) * S.PX[x] + th * S.PXnew[x];
    S.alpha[x] = S.alphanew[x];
  }
}

__global__ void __launch_bounds__(1024)
k_apply(DevState S, const CellDesc* __restrict__ cells, int begin) {
  apply_body(S, cells[begin + blockIdx.x], blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(1024)
k_apply_multi(const DevState* __restrict__ states, const CellRef* __restrict__ refs, int part) {
  __shared__ DevState sS;
  const CellRef rf = refs[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(states + rf.inst);
    int* dst = reinterpret_cast<int*>(&sS);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  // one CTA per cell here (a batch has thousands of cells): the four quadrants in turn
  for (int q = 0; q < 4; ++q) {
    apply_body(sS, sS.cells[part][rf.cell], rf.pos, q);
    __syncthreads();
  }
}

// ============================================================ arena compaction
// Exclusive scan of the box sizes (one block), new offsets into `newoff`.
__device__ __forceinline__ void scan_boxes_body(const DevState& S, long long* newoff) {
  __shared__ long long part[1024];
  const int nb = S.nbasic, tid = threadIdx.x, per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
  long long acc = 0;
  for (int i = b0; i < b1; ++i) acc += (long long)S.box[i].H * S.box[i].W;
  part[tid] = acc;
  __syncthreads();
  if (tid == 0) {
    long long run = 0;
    for (int t = 0; t < (int)blockDim.x; ++t) { long long v = part[t]; part[t] = run; run += v; }
    newoff[nb] = run;
  }
  __syncthreads();
  long long run = part[tid];
  for (int i = b0; i < b1; ++i) { newoff[i] = run; run += (long long)S.box[i].H * S.box[i].W; }
}

__global__ void __launch_bounds__(1024) k_scan_boxes(DevState S, long long* newoff) { scan_boxes_body(S, newoff); }

__device__ __forceinline__ void copy_box_body(const DevState& S, const long long* newoff, int i) {
  const int cur = *S.cur;
  const double* src = S.arena[cur];
  double* dst = S.arena[1 - cur];
  BoxRec b = S.box[i];
  long long sz = (long long)b.H * b.W, no = newoff[i];
  for (long long u = threadIdx.x; u < sz; u += blockDim.x) dst[no + u] = src[b.off + u];
  __syncthreads();
  if (threadIdx.x == 0) S.box[i].off = no;
}

__global__ void __launch_bounds__(256) k_copy_boxes(DevState S, const long long* newoff) {
  copy_box_body(S, newoff, blockIdx.x);
}

__global__ void k_flip_arena(DevState S, const long long* newoff) {
  *S.cur = 1 - *S.cur;
  *S.head = (unsigned long long)newoff[S.nbasic];
}

__global__ void __launch_bounds__(1024) k_scan_boxes_multi(const DevState* __restrict__ states) {
  const DevState& S = states[blockIdx.x];
  scan_boxes_body(S, S.newoff);
}

__global__ void __launch_bounds__(256) k_copy_boxes_multi(const DevState* __restrict__ states) {
  const DevState& S = states[blockIdx.y];
  for (int i = blockIdx.x; i < S.nbasic; i += gridDim.x) {
    copy_box_body(S, S.newoff, i);
    __syncthreads();
  }
}

__global__ void k_flip_arena_multi(const DevState* __restrict__ states, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const DevState& S = states[k];
  *S.cur = 1 - *S.cur;
  *S.head = (unsigned long long)S.newoff[S.nbasic];
}

// ============================================================ inputs and init
__global__ void k_prepare_inputs(const double* mu, const double* nu, double* logmu, double* lognu,
                                 int n, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double a = mu[i], b = nu[i];
    if (!(a > 0.0) || !(b > 0.0) || isinf(a) || isinf(b)) atomicOr(status, ST_BADINPUT);
    logmu[i] = log(a);
    lognu[i] = log(b);
  }
}

// Per basic cell: |mu_i|, the first two moments of mu_i (for <c, mu_i x nu>)
// and |mu_i| |nu|.  One block per basic cell.
__global__ void __launch_bounds__(256)
k_basic_masses(DevState S, const double* nu_mom, double* mumass) {
  __shared__ double red[33 * 4];
  const int i = blockIdx.x, s = S.s, I = i / S.nb, J = i % S.nb;
  double v[4] = {0, 0, 0, 0};
  for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
    int r = I * s + t / s, c = J * s + t % s;
    double m = S.mu[r * S.N + c], x1 = r * S.h, x2 = c * S.h;
    v[0] += m; v[1] += m * x1; v[2] += m * x2; v[3] += m * (x1 * x1 + x2 * x2);
  }
  block_sum<4>(v, red);
  if (threadIdx.x == 0) {
    // nu_mom = (|nu|, sum y1 nu, sum y2 nu, sum |y|^2 nu)
    mumass[i] = v[0];
    S.muinu[i] = v[0] * nu_mom[0];
    // <c, mu_i x nu> = |nu| sum|x|^2 mu - 2 sum x mu . sum y nu + |mu_i| sum |y|^2 nu
    S.Cc[i] = nu_mom[0] * v[3] - 2.0 * (v[1] * nu_mom[1] + v[2] * nu_mom[2]) + v[0] * nu_mom[3];
    S.Hh[i] = 0.0;
  }
}

__global__ void __launch_bounds__(512) k_moments(const double* nu, int N, double h, double* out) {
  __shared__ double red[33 * 4];
  double v[4] = {0, 0, 0, 0};
  for (int y = threadIdx.x; y < N * N; y += blockDim.x) {
    double m = nu[y], y1 = (y / N) * h, y2 = (y % N) * h;
    v[0] += m; v[1] += m * y1; v[2] += m * y2; v[3] += m * (y1 * y1 + y2 * y2);
  }
  block_sum<4>(v, red);
  if (threadIdx.x == 0) for (int k = 0; k < 4; ++k) out[k] = v[k];
}

// Product plan pi0 = mu x nu: nu_i = |mu_i| nu on the full grid, truncated.
// Pass 1 (mode 0): tight box of the kept entries.  Pass 2 (mode 1): values, P_Y.
__global__ void __launch_bounds__(256)
k_init_product(DevState S, const double* mumass, int mode) {
  __shared__ int bb[4];
  const int i = blockIdx.x, N = S.N, n = N * N;
  const double mi = mumass[i];
  double* arena = S.arena[*S.cur];
  if (mode == 0) {
    if (threadIdx.x == 0) { bb[0] = 1 << 30; bb[1] = -1; bb[2] = 1 << 30; bb[3] = -1; }
    __syncthreads();
    int lb[4] = {1 << 30, -1, 1 << 30, -1};
    for (int y = threadIdx.x; y < n; y += blockDim.x) {
      if (mi * S.nu[y] >= S.thr) {
        int k = y / N, l = y % N;
        lb[0] = min(lb[0], k); lb[1] = max(lb[1], k); lb[2] = min(lb[2], l); lb[3] = max(lb[3], l);
      }
    }
    lb[0] = warp_min(lb[0]); lb[1] = warp_max(lb[1]); lb[2] = warp_min(lb[2]); lb[3] = warp_max(lb[3]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bb[0], lb[0]); atomicMax(&bb[1], lb[1]); atomicMin(&bb[2], lb[2]); atomicMax(&bb[3], lb[3]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      BoxRec b = {0, 0, 0, 0, 0};
      if (bb[1] >= 0) { b.k0 = bb[0]; b.l0 = bb[2]; b.H = bb[1] - bb[0] + 1; b.W = bb[3] - bb[2] + 1; }
      S.box[i] = b;
    }
  } else {
    BoxRec b = S.box[i];
    for (int u = threadIdx.x; u < b.H * b.W; u += blockDim.x) {
      int y = (b.k0 + u / b.W) * N + b.l0 + u % b.W;
      double v = mi * S.nu[y];
      if (v < S.thr) v = 0.0;
      arena[b.off + u] = v;
      if (v != 0.0) atomicAdd(S.PY + y, v);
    }
  }
}

__global__ void k_set_offsets(DevState S, const long long* newoff) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nbasic; i += gridDim.x * blockDim.x)
    S.box[i].off = newoff[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) *S.head = (unsigned long long)newoff[S.nbasic];
}

__global__ void k_px_product(DevState S, const double* nu_mom) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < S.N * S.N; x += gridDim.x * blockDim.x) {
    S.PX[x] = S.mu[x] * nu_mom[0];
    S.alpha[x] = 0.0;
  }
}

// g[y] = log nu(y) + beta0(y)/eps0 in float (the test pass of k_init_duals).
__global__ void k_log_nu_beta(const double* __restrict__ lognu, const double* __restrict__ beta0, double eps0,
                              int n, float* __restrict__ g) {
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x)
    g[y] = (float)(lognu[y] + beta0[y] / eps0);
}

// Plan from duals pi = exp((alpha0 + beta0 - c)/eps0) mu x nu, per basic cell.
// mode 0: tight box of {y : nu_i(y) >= thr} from the full-grid log marginal,
//         two 1-D log-sum-exp passes over X_i: the first in FP64 (s N values),
//         the second over every y of the grid first in float (gf = the float
//         log nu + beta0/eps0); only where the float value lies within a
//         safety band of log thr (its float error is ~1e-2 at |values| ~ 1e5)
//         is the FP64 value computed and compared, so the box is the one of
//         the FP64 test;
// mode 1: values on the box (dense over X_i), C_i, H_i, P_Y.
constexpr int kInitChunk = 128;   // box columns per pass of the dual-initialised fill
constexpr int kInitBand = 2048;   // band pixels listed per basic cell by the box test
__global__ void __launch_bounds__(1024)
k_init_duals(DevState S, const double* __restrict__ alpha0, const double* __restrict__ beta0,
             double eps0, int mode, const float* __restrict__ gf) {
  extern __shared__ double tsm[];   // mode 0: see init_box_smem; mode 1: 3 s kInitChunk doubles
  __shared__ int bb[4];
  __shared__ double red[33 * 2];
  const int i = blockIdx.x, s = S.s, N = S.N, I = i / S.nb, J = i % S.nb;
  const int r0 = I * s, c0 = J * s;
  const double q = S.h * S.h / eps0;
  double* arena = S.arena[*S.cur];
  if (mode == 0) {
    // shared: T(r, l) in double (only the columns flagged below) | T in float | X values in
    // float | column flags | list of the pixels in the band of the float test
    float* tsmf = reinterpret_cast<float*>(tsm + s * N);
    float* xvf = tsmf + s * N;
    unsigned char* colflag = reinterpret_cast<unsigned char*>(xvf + s * s);
    int* band = reinterpret_cast<int*>(colflag + ((N + 15) & ~15));
    __shared__ int nband;
    const double ie0 = 1.0 / eps0;
    const float qf = (float)q, L2E = (float)DD_LOG2E, LN2 = (float)DD_LN2;
    for (int t = threadIdx.x; t < s * s; t += blockDim.x) {
      const int x = (r0 + t / s) * N + c0 + t % s;
      xvf[t] = (float)(alpha0[x] * ie0 + S.logmu[x]);
    }
    for (int l = threadIdx.x; l < N; l += blockDim.x) colflag[l] = 0;
    if (threadIdx.x == 0) { nband = 0; bb[0] = 1 << 30; bb[1] = -1; bb[2] = 1 << 30; bb[3] = -1; }
    __syncthreads();
    // float T(r, l) = log sum_{c in cols(X_i)} exp(alpha0/eps0 + log mu - q (c - l)^2)
    for (int t = threadIdx.x; t < s * N; t += blockDim.x) {
      const int r = t / N, l = t - (t / N) * N;
      float mx = -INFINITY;
      for (int c = 0; c < s; ++c) {
        const float d = (float)(c0 + c - l);
        mx = fmaxf(mx, xvf[r * s + c] - qf * d * d);
      }
      float acc = 0.0f;
      for (int c = 0; c < s; ++c) {
        const float d = (float)(c0 + c - l);
        acc += dd_ex2((xvf[r * s + c] - qf * d * d - mx) * L2E);
      }
      tsmf[t] = mx + dd_lg2(acc) * LN2;
    }
    __syncthreads();
    int lb[4] = {1 << 30, -1, 1 << 30, -1};
    const double lthr = log(S.thr);
    const float lthrf = (float)lthr;
    auto keep = [&](int k, int l) {
      lb[0] = min(lb[0], k); lb[1] = max(lb[1], k); lb[2] = min(lb[2], l); lb[3] = max(lb[3], l);
    };
    // the float test of every pixel; `band` collects those it cannot decide
    for (int y = threadIdx.x; y < N * N; y += blockDim.x) {
      const int k = y / N, l = y - (y / N) * N;
      float mxf = -INFINITY, big = fabsf(gf[y]);
      for (int r = 0; r < s; ++r) {
        const float d = (float)(r0 + r - k), v = tsmf[r * N + l];
        mxf = fmaxf(mxf, v - qf * d * d);
        big = fmaxf(big, fabsf(v) + qf * d * d);
      }
      // float value and its error bound (a few ulps of the magnitudes that cancel; the
      // float X values and T add ~1e-7 of the same magnitudes)
      const float band_w = 0.5f + 1e-5f * big;
      const float lo = gf[y] + mxf;   // log nu_i(y) lies in [lo, lo + log s]
      if (lo + dd_lg2((float)s) * LN2 < lthrf - band_w) continue;   // clearly below the threshold
      float accf = 0.0f;
      for (int r = 0; r < s; ++r) {
        const float d = (float)(r0 + r - k);
        accf += dd_ex2((tsmf[r * N + l] - qf * d * d - mxf) * L2E);
      }
      const float lvf = lo + dd_lg2(accf) * LN2;
      if (lvf >= lthrf + band_w) {
        keep(k, l);
      } else if (lvf > lthrf - band_w) {
        colflag[l] = 1;
        const int j = atomicAdd(&nband, 1);
        if (j < kInitBand) band[j] = y;
      }
    }
    __syncthreads();
    // double T on the flagged columns
    for (int t = threadIdx.x; t < s * N; t += blockDim.x) {
      const int r = t / N, l = t - (t / N) * N;
      if (!colflag[l]) continue;
      double mx = -INFINITY;
      for (int c = 0; c < s; ++c) {
        const int x = (r0 + r) * N + c0 + c;
        const double d = c0 + c - l;
        mx = fmax(mx, alpha0[x] * ie0 + S.logmu[x] - q * d * d);
      }
      double acc = 0.0;
      for (int c = 0; c < s; ++c) {
        const int x = (r0 + r) * N + c0 + c;
        const double d = c0 + c - l;
        acc += exp(alpha0[x] * ie0 + S.logmu[x] - q * d * d - mx);
      }
      tsm[t] = mx + log(acc);
    }
    __syncthreads();
    // the double test of the band pixels (rescanning all pixels if the list overflowed)
    auto dtest = [&](int y) {
      const int k = y / N, l = y - (y / N) * N;
      double mx = -INFINITY;
      for (int r = 0; r < s; ++r) { const double d = r0 + r - k; mx = fmax(mx, tsm[r * N + l] - q * d * d); }
      double acc = 0.0;
      for (int r = 0; r < s; ++r) { const double d = r0 + r - k; acc += exp(tsm[r * N + l] - q * d * d - mx); }
      if (S.lognu[y] + beta0[y] * ie0 + mx + log(acc) >= lthr) keep(k, l);
    };
    const int nb = nband;
    if (nb <= kInitBand) {
      for (int j = threadIdx.x; j < nb; j += blockDim.x) dtest(band[j]);
    } else {
      for (int y = threadIdx.x; y < N * N; y += blockDim.x) {
        const int k = y / N, l = y - (y / N) * N;
        if (!colflag[l]) continue;
        float mxf = -INFINITY, big = fabsf(gf[y]);
        for (int r = 0; r < s; ++r) {
          const float d = (float)(r0 + r - k), v = tsmf[r * N + l];
          mxf = fmaxf(mxf, v - qf * d * d);
          big = fmaxf(big, fabsf(v) + qf * d * d);
        }
        const float band_w = 0.5f + 1e-5f * big;
        const float lo = gf[y] + mxf;
        if (lo + dd_lg2((float)s) * LN2 < lthrf - band_w) continue;
        float accf = 0.0f;
        for (int r = 0; r < s; ++r) {
          const float d = (float)(r0 + r - k);
          accf += dd_ex2((tsmf[r * N + l] - qf * d * d - mxf) * L2E);
        }
        const float lvf = lo + dd_lg2(accf) * LN2;
        if (lvf < lthrf + band_w && lvf > lthrf - band_w) dtest(y);
      }
    }
    lb[0] = warp_min(lb[0]); lb[1] = warp_max(lb[1]); lb[2] = warp_min(lb[2]); lb[3] = warp_max(lb[3]);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&bb[0], lb[0]); atomicMax(&bb[1], lb[1]); atomicMin(&bb[2], lb[2]); atomicMax(&bb[3], lb[3]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      BoxRec b = {0, 0, 0, 0, 0};
      if (bb[1] >= 0) { b.k0 = bb[0]; b.l0 = bb[2]; b.H = bb[1] - bb[0] + 1; b.W = bb[3] - bb[2] + 1; }
      S.box[i] = b;
    }
  } else {
    // Separable evaluation on the box (|x - y|^2 splits over the axes), in
    // column chunks of kInitChunk: per row r of X_i and column l of the chunk
    //   T1(r, l) = log sum_c exp(alpha0/eps0 + log mu - q (c - l)^2)  (c over the columns of X_i)
    // with the conditional means of (c - l)^2 and alpha0/eps0 under those terms;
    // per box point y = (k, l) the sum over the rows r of X_i then gives
    //   nu_i(y) = nu(y) exp(beta0/eps0) sum_r exp(T1 - q (r - k)^2),
    //   sum_x c pi = h^2 sum_r w_r ((r - k)^2 + E[(c - l)^2]),  sum_x pi log(pi / mu nu) likewise.
    // s exponentials per box point instead of s^2.
    double* T1 = tsm;
    double* M2 = T1 + s * kInitChunk;
    double* MA = M2 + s * kInitChunk;
    const BoxRec b = S.box[i];
    double v[2] = {0.0, 0.0};
    const double ie0 = 1.0 / eps0;
    for (int lc = 0; lc < b.W; lc += kInitChunk) {
      const int wc = min(kInitChunk, b.W - lc);
      for (int t = threadIdx.x; t < s * wc; t += blockDim.x) {
        const int r = t / wc, l = b.l0 + lc + t % wc;
        double mx = -INFINITY;
        for (int c = 0; c < s; ++c) {
          const int x = (r0 + r) * N + c0 + c;
          const double d = c0 + c - l;
          mx = fmax(mx, alpha0[x] * ie0 + S.logmu[x] - q * d * d);
        }
        double a = 0.0, a2 = 0.0, aa = 0.0;
        for (int c = 0; c < s; ++c) {
          const int x = (r0 + r) * N + c0 + c;
          const double d = c0 + c - l;
          const double w = exp(alpha0[x] * ie0 + S.logmu[x] - q * d * d - mx);
          a += w; a2 += w * d * d; aa += w * (alpha0[x] * ie0);
        }
        T1[r * kInitChunk + t % wc] = mx + log(a);
        M2[r * kInitChunk + t % wc] = a2 / a;
        MA[r * kInitChunk + t % wc] = aa / a;
      }
      __syncthreads();
      for (int u = threadIdx.x; u < b.H * wc; u += blockDim.x) {
        const int kk = u / wc, lj = u % wc;
        const int k = b.k0 + kk, l = b.l0 + lc + lj, y = k * N + l;
        double mx = -INFINITY;
        for (int r = 0; r < s; ++r) {
          const double d = r0 + r - k;
          mx = fmax(mx, T1[r * kInitChunk + lj] - q * d * d);
        }
        double a = 0.0, ac = 0.0, aa = 0.0;
        for (int r = 0; r < s; ++r) {
          const double d = r0 + r - k;
          const double w = exp(T1[r * kInitChunk + lj] - q * d * d - mx);
          a += w; ac += w * (d * d + M2[r * kInitChunk + lj]); aa += w * MA[r * kInitChunk + lj];
        }
        const double by = beta0[y] * ie0;
        const double acc = S.nu[y] * exp(by + mx) * a;   // nu_i(y) = sum_x pi(x, y)
        const double val = acc < S.thr ? 0.0 : acc;
        arena[b.off + kk * b.W + lc + lj] = val;
        if (val != 0.0) atomicAdd(S.PY + y, val);
        const double cc = S.h * S.h * ac / a;   // E[c] under pi(., y)
        v[0] += cc * acc;
        // sum_x pi (log(pi / (mu nu)) - 1), log(pi / (mu nu)) = (alpha0 + beta0 - c)/eps0
        v[1] += acc * (aa / a + by - cc * ie0 - 1.0);
      }
      __syncthreads();
    }
    block_sum<2>(v, red);
    if (threadIdx.x == 0) {
      S.Cc[i] = v[0];
      S.Hh[i] = v[1] + S.muinu[i];
    }
  }
}

// ================================================================ reductions
// out: [sum_i (C_i + eps H_i), lam KL(P_X|mu), lam KL(P_Y|nu), |P_Y|, box entries]
__global__ void __launch_bounds__(512) k_score(DevState S, double* out) {
  __shared__ double red[33 * 5];
  const int n = S.N * S.N;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, dt = gridDim.x * blockDim.x;
  double v[5] = {0, 0, 0, 0, 0};
  for (int y = t0; y < n; y += dt) {
    v[1] += S.lam * dd_kl_term(S.PX[y], S.mu[y]);
    v[2] += S.lam * dd_kl_term(S.PY[y], S.nu[y]);
    v[3] += S.PY[y];
  }
  for (int i = t0; i < S.nbasic; i += dt) {
    v[0] += S.Cc[i] + S.eps * S.Hh[i];
    v[4] += (double)S.box[i].H * S.box[i].W;
  }
  block_sum_to<5>(v, red, out);
}

// out[k] = sum over g of partials[g * K + k], g in order.
__global__ void k_sum_partials(const double* partials, int G, int K, double* out) {
  const int k = threadIdx.x;
  if (k >= K) return;
  double a = 0.0;
  for (int g = 0; g < G; ++g) a += partials[g * K + k];
  out[k] = a;
}

// Dual value and marginal errors of the certificate.
// z: log int exp((alpha - c)/eps) dmu per y (natural units); beta* = -kappa z.
// out: [sum_y nu e^{beta*/eps + z}, sum_x (e^{-alpha/lam}-1) mu, sum_y (e^{-beta*/lam}-1) nu,
//       |mu|, |nu|, L1 X error, L1 Y error]
__global__ void __launch_bounds__(512)
k_cert(DevState S, const double* z, double* beta_out, double* out) {
  __shared__ double red[33 * 7];
  const int n = S.N * S.N;
  const double eps = S.eps, lam = S.lam, kap = eps / (1.0 + eps / lam);
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
    double b = -kap * z[y];
    if (beta_out) beta_out[y] = b;
    double ea = exp(-S.alpha[y] / lam), eb = exp(-b / lam);
    v[0] += S.nu[y] * exp(b / eps + z[y]);
    v[1] += (ea - 1.0) * S.mu[y];
    v[2] += (eb - 1.0) * S.nu[y];
    v[3] += S.mu[y];
    v[4] += S.nu[y];
    v[5] += fabs(S.PX[y] - ea * S.mu[y]);
    v[6] += fabs(S.PY[y] - eb * S.nu[y]);
  }
  block_sum_to<7>(v, red, out);
}

// ======================================================= host launch wrappers
cudaError_t launch_decide(const DevState& S, const CellDesc* cells, int begin, int nbatch, cudaStream_t st) {
  int nblk = kRedBlocks;
  int n = S.N * S.N;
  if (n < nblk * 512) nblk = (n + 511) / 512;
  if (nblk < 1) nblk = 1;
  k_decide<<<nblk, 512, 0, st>>>(S, cells, begin, nbatch);
  return cudaGetLastError();
}
// The search of GetWeights_line after k_decide: one evaluation at 1 and lo,
// then up to kLineIters evaluations (no-ops once the search has stopped).
cudaError_t launch_line_search(const DevState& S, const CellDesc* cells, int begin, int nbatch, double* partials,
                               cudaStream_t st) {
  int G = (S.N * S.N + 511) / 512;
  if (G < nbatch) G = nbatch;
  if (G > kRedBlocks) G = kRedBlocks;
  for (int k = 0; k <= kLineIters; ++k) {
    k_line_eval<<<G, 512, 0, st>>>(S, cells, begin, nbatch, k == 0, partials);
    k_sum_partials<<<1, 32, 0, st>>>(partials, G, 4, S.line + 12);
    k_line_step<<<1, 32, 0, st>>>(S, k == 0, k == kLineIters);
  }
  return cudaGetLastError();
}
cudaError_t launch_decide_multi(const DevState* states, int ninst, int maxn, int part, int sub, cudaStream_t st) {
  int nblk = (maxn * maxn + 511) / 512;
  if (nblk > kRedBlocks) nblk = kRedBlocks;
  if (nblk < 1) nblk = 1;
  k_decide_multi<<<dim3(nblk, ninst), 512, 0, st>>>(states, part, sub);
  return cudaGetLastError();
}
cudaError_t launch_apply_multi(const DevState* states, const CellRef* refs, int nref, int part, cudaStream_t st) {
  if (nref > 0) k_apply_multi<<<nref, 1024, 0, st>>>(states, refs, part);
  return cudaGetLastError();
}
cudaError_t launch_compact_multi(const DevState* states, int ninst, int max_nbasic, cudaStream_t st) {
  k_scan_boxes_multi<<<ninst, 1024, 0, st>>>(states);
  k_copy_boxes_multi<<<dim3(max_nbasic < 4096 ? max_nbasic : 4096, ninst), 256, 0, st>>>(states);
  k_flip_arena_multi<<<(ninst + 127) / 128, 128, 0, st>>>(states, ninst);
  return cudaGetLastError();
}
cudaError_t launch_apply(const DevState& S, const CellDesc* cells, int begin, int nbatch, cudaStream_t st) {
  k_apply<<<dim3(nbatch, 4), 1024, 0, st>>>(S, cells, begin);
  return cudaGetLastError();
}
cudaError_t launch_compact(const DevState& S, long long* newoff, cudaStream_t st) {
  k_scan_boxes<<<1, 1024, 0, st>>>(S, newoff);
  k_copy_boxes<<<S.nbasic, 256, 0, st>>>(S, newoff);
  k_flip_arena<<<1, 1, 0, st>>>(S, newoff);
  return cudaGetLastError();
}
cudaError_t launch_prepare_inputs(const double* mu, const double* nu, double* logmu, double* lognu,
                                  int n, int* status, cudaStream_t st) {
  k_prepare_inputs<<<(n + 255) / 256, 256, 0, st>>>(mu, nu, logmu, lognu, n, status);
  return cudaGetLastError();
}
__global__ void k_px_duals(DevState S, const double* alpha0, const double* w, double eps0) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < S.N * S.N; x += gridDim.x * blockDim.x) {
    S.PX[x] = S.mu[x] * exp(alpha0[x] / eps0 + w[x]);
    S.alpha[x] = alpha0[x];
  }
}

__global__ void __launch_bounds__(256) k_copy_boxes_to(DevState S, const long long* newoff, double* dst) {
  const int i = blockIdx.x;
  const double* src = S.arena[*S.cur];
  BoxRec b = S.box[i];
  long long sz = (long long)b.H * b.W, no = newoff[i];
  for (long long u = threadIdx.x; u < sz; u += blockDim.x) dst[no + u] = src[b.off + u];
}

__global__ void k_reset_cur(DevState S, const long long* newoff) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.nbasic; i += gridDim.x * blockDim.x)
    S.box[i].off = newoff[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *S.cur = 0;
    *S.head = (unsigned long long)newoff[S.nbasic];
  }
}

cudaError_t launch_init_product_boxes(const DevState& S, double* nu_mom, double* mumass, long long* newoff,
                                      cudaStream_t st) {
  k_moments<<<1, 512, 0, st>>>(S.nu, S.N, S.h, nu_mom);
  k_basic_masses<<<S.nbasic, 256, 0, st>>>(S, nu_mom, mumass);
  k_init_product<<<S.nbasic, 256, 0, st>>>(S, mumass, 0);
  k_scan_boxes<<<1, 1024, 0, st>>>(S, newoff);
  return cudaGetLastError();
}
cudaError_t launch_init_product_fill(const DevState& S, double* nu_mom, double* mumass, long long* newoff,
                                     cudaStream_t st) {
  k_set_offsets<<<(S.nbasic + 255) / 256, 256, 0, st>>>(S, newoff);
  k_init_product<<<S.nbasic, 256, 0, st>>>(S, mumass, 1);
  k_px_product<<<(S.N * S.N + 255) / 256, 256, 0, st>>>(S, nu_mom);
  return cudaGetLastError();
}
// gscratch: N*N floats of device scratch
// dynamic shared memory of the box test (mode 0 of k_init_duals)
static size_t init_box_smem(int s, int N) {
  return (size_t)s * N * (sizeof(double) + sizeof(float)) + (size_t)s * s * sizeof(float) + ((N + 15) & ~15) +
         kInitBand * sizeof(int);
}
cudaError_t launch_init_duals_boxes(const DevState& S, const double* alpha0, const double* beta0, double eps0,
                                    double* nu_mom, double* mumass, long long* newoff, float* gscratch,
                                    cudaStream_t st) {
  k_moments<<<1, 512, 0, st>>>(S.nu, S.N, S.h, nu_mom);
  k_basic_masses<<<S.nbasic, 256, 0, st>>>(S, nu_mom, mumass);
  const int n = S.N * S.N;
  k_log_nu_beta<<<(n + 255) / 256, 256, 0, st>>>(S.lognu, beta0, eps0, n, gscratch);
  const size_t sm = init_box_smem(S.s, S.N);
  cudaFuncSetAttribute(k_init_duals, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_init_duals<<<S.nbasic, 1024, sm, st>>>(S, alpha0, beta0, eps0, 0, gscratch);
  k_scan_boxes<<<1, 1024, 0, st>>>(S, newoff);
  return cudaGetLastError();
}
cudaError_t launch_init_duals_fill(const DevState& S, const double* alpha0, const double* beta0, double eps0,
                                   const double* w, long long* newoff, cudaStream_t st) {
  k_set_offsets<<<(S.nbasic + 255) / 256, 256, 0, st>>>(S, newoff);
  const size_t sm = 3 * sizeof(double) * (size_t)S.s * kInitChunk;
  cudaFuncSetAttribute(k_init_duals, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(sm, init_box_smem(S.s, S.N)));
  k_init_duals<<<S.nbasic, 256, sm, st>>>(S, alpha0, beta0, eps0, 1, nullptr);
  k_px_duals<<<(S.N * S.N + 255) / 256, 256, 0, st>>>(S, alpha0, w, eps0);
  return cudaGetLastError();
}
cudaError_t launch_regrow(const DevState& S, double* new0, double* new1, long long* newoff, cudaStream_t st) {
  (void)new1;
  k_scan_boxes<<<1, 1024, 0, st>>>(S, newoff);
  k_copy_boxes_to<<<S.nbasic, 256, 0, st>>>(S, newoff, new0);
  k_reset_cur<<<(S.nbasic + 255) / 256, 256, 0, st>>>(S, newoff);
  return cudaGetLastError();
}
// partials: kRedBlocks * 8 doubles of scratch (NULL: one block)
cudaError_t launch_score(const DevState& S, double* out, cudaStream_t st, double* partials) {
  const int G = red_blocks((long long)S.N * S.N, 512, partials);
  if (G == 1) {
    k_score<<<1, 512, 0, st>>>(S, out);
  } else {
    k_score<<<G, 512, 0, st>>>(S, partials);
    k_sum_partials<<<1, 32, 0, st>>>(partials, G, 5, out);
  }
  return cudaGetLastError();
}
cudaError_t launch_cert(const DevState& S, const double* z, double* beta_out, double* out, cudaStream_t st,
                        double* partials) {
  const int G = red_blocks((long long)S.N * S.N, 512, partials);
  if (G == 1) {
    k_cert<<<1, 512, 0, st>>>(S, z, beta_out, out);
  } else {
    k_cert<<<G, 512, 0, st>>>(S, z, beta_out, partials);
    k_sum_partials<<<1, 32, 0, st>>>(partials, G, 7, out);
  }
  return cudaGetLastError();
}
