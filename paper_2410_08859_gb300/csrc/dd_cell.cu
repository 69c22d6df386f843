// Cell subproblem kernel: one CTA per composite cell of a sub-batch.
//
// For cell J with X box X_J (nx1 x nx2 pixels) and Y box B_J (H x W pixels):
//  a1  rho = max(0, P_Y pi - nu_J)/nu on B_J             (Section 5.1, "Computing and handling nu_{-J}")
//  a2  X-half  alpha = -(eps lam/(eps+lam)) log int exp((beta-c)/eps) dnu   (Eq. sinkhorn-X-iteration)
//  a3  Y-half  per y the root of log(rho + e^{beta/eps + z}) + beta/lam = 0 (Eq. proxdiv-problem)
//  a4  stop when PD/lam = KL(P_X pi | e^{-alpha/lam} mu_J) <= err |mu_J|   (Eq. PD-gap-KL)
//  a5  nu~_i(y), C~_i = <c, pi~_i>, H~_i = KL(pi~_i | mu_i x nu) of the new cell plan per
//      member basic cell i, P_X pi~ and the KL_X change for the step-size decision.
//
// GB300 design:
//  * Everything a cell iterates on lives in shared memory; the cost is never stored: c/eps is
//    q |xi - eta|^2 with integer pixel offsets and q = h^2/eps.
//  * |x - y|^2 separates over the two axes, so every log-sum-exp over a rectangle is computed as
//    two 1-D passes (rows, then columns): (nx1 nx2 W + nx1 H W) terms instead of nx1 nx2 H W.
//  * Cell-local frames keep float arithmetic accurate: with x_c, y_c the box centres and
//    D = x_c - y_c (integer), alpha/eps = A + a(xi) + 2 q D.xi and beta/eps = B + b(eta) - 2 q D.eta
//    with A, B per-cell doubles and B = q|D|^2 - A, so that (alpha + beta - c)/eps =
//    a(xi) + b(eta) - q |xi - eta|^2 exactly; a and b stay moderate while alpha/eps is ~1e4-1e5.
//  * exp/log are ex2.approx/lg2.approx in log2 units; each 1-D log-sum-exp is shifted by the
//    previous iteration's value (one pass), with an exact max-shifted fallback.
#include <cooperative_groups.h>

#include <algorithm>

#include "dd_common.cuh"

// Threads per CTA of the cell kernels (the cell body works with any multiple
// of 32 up to 1024; the block reductions assume at most 32 warps).
#ifndef DD_CELL_THREADS
#define DD_CELL_THREADS 512
#endif
constexpr int kCellThreads = DD_CELL_THREADS;

namespace {

template <typename R, typename F>
__device__ __forceinline__ R lse2_1d(F src, int M, R ctr, R q2, R shift, bool use_shift) {
  // log2 sum_m 2^{src(m) - q2 (m - ctr)^2}
  if (use_shift) {
    R a0 = R(0), a1 = R(0);
    R d = -ctr;
    int m = 0;
    for (; m + 1 < M; m += 2) {
      R v0 = src(m) - q2 * d * d - shift;
      d += R(1);
      R v1 = src(m + 1) - q2 * d * d - shift;
      d += R(1);
      a0 += dd_ex2(v0);
      a1 += dd_ex2(v1);
    }
    if (m < M) a0 += dd_ex2(src(m) - q2 * d * d - shift);
    R acc = a0 + a1;
    if (acc > R(1e-25) && acc < R(1e25)) return shift + dd_lg2(acc);
  }
  R mx = -dd_inf<R>();
  R d = -ctr;
  for (int m = 0; m < M; ++m, d += R(1)) mx = max(mx, src(m) - q2 * d * d);
  if (!(mx > -dd_inf<R>())) return mx;
  R acc = R(0);
  d = -ctr;
  for (int m = 0; m < M; ++m, d += R(1)) acc += dd_ex2(src(m) - q2 * d * d - mx);
  return mx + dd_lg2(acc);
}

// One pass of the epilogue statistics against the shift sh: over m in [b, e),
// with d = m - ctr and w = 2^{src(m) - q2 d^2 - sh}, the sums of w,
// w (A(m) - qR d^2) and w ((d + D)^2 + B(m)).
template <typename R, typename F, typename GA, typename GB>
__device__ __forceinline__ void moments_pass(F src, GA A, GB B, R qR, R D, int b, int e, R ctr, R q2, R sh, R& sw,
                                             R& sa, R& sd) {
  sw = sa = sd = R(0);
  R d = R(b) - ctr;
  for (int m = b; m < e; ++m, d += R(1)) {
    const R w = dd_ex2(src(m) - q2 * d * d - sh);
    sw += w;
    sa += w * (A(m) - qR * d * d);
    sd += w * ((d + D) * (d + D) + B(m));
  }
}

// Epilogue statistics of one target over the sources m in [b, e): with
// v_m = src(m) - q2 (m - ctr)^2 (log2 units) returns L = log2 sum_m 2^{v_m} and
// the means m1 = <A(m) - qR d^2>, m2 = <(d + D)^2 + B(m)> under the weights
// 2^{v_m - L} (d = m - ctr).  With use_shift, `shift` is an upper bound of L
// (the full-range log-sum-exp of the same terms): one pass of exponentials
// against it, and only if that sum leaves [1e-30, 1e30] (the sub-range holds a
// negligible share) the exact pass against the maximum.  Without a shift the
// maximum is found first.
template <typename R, typename F, typename GA, typename GB>
__device__ __forceinline__ R lse_moments(F src, GA A, GB B, R qR, R D, int b, int e, R ctr, R q2, R shift,
                                         bool use_shift, R& m1, R& m2) {
  auto maxpass = [&]() {
    R mx = -dd_inf<R>();
    R d = R(b) - ctr;
    for (int m = b; m < e; ++m, d += R(1)) mx = max(mx, src(m) - q2 * d * d);
    return mx;
  };
  R sh = shift;
  if (!use_shift) {
    sh = maxpass();
    if (!(sh > -dd_inf<R>())) {
      m1 = m2 = R(0);
      return sh;
    }
  }
  for (int pass = 0;; ++pass) {
    R sw, sa, sd;
    moments_pass<R>(src, A, B, qR, D, b, e, ctr, q2, sh, sw, sa, sd);
    if (!use_shift || pass == 1 || (sw >= R(1e-30) && sw <= R(1e30))) {
      const R isw = R(1) / sw;
      m1 = sa * isw;
      m2 = sd * isw;
      return sh + dd_lg2(sw);
    }
    // the shift was far from L: the exact pass against the maximum
    sh = maxpass();
    if (!(sh > -dd_inf<R>())) {
      m1 = m2 = R(0);
      return sh;
    }
  }
}

// Partial sum of 2^{src(m) - q2 (m - ctr)^2 - shift} over m = part, part + P, ...
// (eight independent accumulators to keep several ex2 in flight).
template <typename R, typename F>
__device__ __forceinline__ R psum2(F src, int M, R ctr, R q2, R shift, int part, int P) {
  R a[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
  const R dP = R(P);
  R d = R(part) - ctr;
  int m = part;
  for (; m + 7 * P < M; m += 8 * P) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const R dk = d + R(k) * dP;
      a[k] += dd_ex2(src(m + k * P) - q2 * dk * dk - shift);
    }
    d += R(8) * dP;
  }
  for (; m < M; m += P, d += dP) a[0] += dd_ex2(src(m) - q2 * d * d - shift);
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

template <typename R, typename F>
__device__ __forceinline__ R pmax2(F src, int M, R ctr, R q2, int part, int P) {
  R mx = -dd_inf<R>();
  const R dP = R(P);
  R d = R(part) - ctr;
  for (int m = part; m < M; m += P, d += dP) mx = max(mx, src(m) - q2 * d * d);
  return mx;
}

// log2 sum_m 2^{src(m) - q2 (m - ctr)^2} computed by the P lanes of an aligned
// lane group (P a power of two dividing 32).  Must be called by all 32 lanes of
// the warp.  With use_shift the sum is taken against `shift` (the previous
// iteration's value) in one pass; if the group's sum leaves the safe range, or
// without a shift, the warp falls back to the exact max-shifted two passes.
template <typename R, typename F>
__device__ __forceinline__ R lse2_group(F src, int M, R ctr, R q2, R shift, bool use_shift, int part, int P) {
  R acc = R(0);
  bool bad = true;
  if (use_shift) {
    acc = psum2<R>(src, M, ctr, q2, shift, part, P);
    for (int o = 1; o < P; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    bad = !(acc > R(1e-25) && acc < R(1e25));
  }
  if (__any_sync(0xffffffffu, bad)) {
    R mx = pmax2<R>(src, M, ctr, q2, part, P);
    for (int o = 1; o < P; o <<= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const bool fin = mx > -dd_inf<R>();
    R s2 = psum2<R>(src, M, ctr, q2, fin ? mx : R(0), part, P);
    for (int o = 1; o < P; o <<= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (bad) return fin ? mx + dd_lg2(s2) : mx;
  }
  return shift + dd_lg2(acc);
}

// Lanes per target for a pass with `nt` targets of `M` sources on `nthr` threads.
__device__ __forceinline__ int lanes_per_target(int nt, int M, int nthr) {
  int P = 1;
  while (P < 32 && nt * P * 2 <= nthr && P * 2 <= M) P *= 2;
  return P;
}

// Root u of g(u) = (1+s) u + c0 + softplus(lr - u) = 0, i.e. of
// log(rho + e^u) + s u + c0 = 0 with lr = log rho (Eq. proxdiv-problem with
// u = beta/eps + z).  g is convex and increasing (g' = 1 + s - sigmoid(lr - u) >= s).
// Both lines (1+s)u + c0 and s u + c0 + lr lie below g, so g >= 0 at
// min(u0, u1), their roots; Newton from there decreases monotonically to the root.
template <typename R>
__device__ __forceinline__ R newton_u(R lr, R c0, R s, int maxit) {
  const R L2E = R(DD_LOG2E), LN2 = R(DD_LN2);
  const R one_s = R(1) + s;
  R u = -c0 / one_s;
  if (!(lr > -dd_inf<R>())) return u;  // rho = 0: closed form (Eq. sinkhorn-iters-ot)
  if (s > R(0)) u = min(u, -(lr + c0) / s);
  const R tol = sizeof(R) == 4 ? R(2e-6) : R(1e-14);
  for (int k = 0; k < maxit; ++k) {
    R t = lr - u;
    R e = dd_ex2(-fabs(t) * L2E);
    R ie = dd_rcp(R(1) + e);
    R sp = max(t, R(0)) + dd_lg2(R(1) + e) * LN2;
    R sig = t >= R(0) ? ie : e * ie;
    R g = one_s * u + c0 + sp;
    R du = g * dd_rcp(one_s - sig);
    u -= du;
    if (fabs(du) <= tol * max(R(1), fabs(u))) break;
  }
  return u;
}

// Two independent roots of newton_u advanced in lock-step (their dependency
// chains interleave; each stops on its own tolerance).  `uw` holds a previous
// root per target (or NaN): one Newton step from it lands right of the root
// (g is convex and increasing), and the start is the smaller of that point and
// the bound min(u0, u1), so the iteration still descends monotonically.
template <typename R>
__device__ __forceinline__ void newton_u2(const R (&lr)[2], const R (&c0)[2], const R (&uw)[2], R s, int maxit,
                                          R (&u)[2]) {
  const R L2E = R(DD_LOG2E), LN2 = R(DD_LN2);
  const R one_s = R(1) + s;
  const R tol = sizeof(R) == 4 ? R(2e-6) : R(1e-14);
  bool act[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    u[k] = -c0[k] / one_s;
    act[k] = lr[k] > -dd_inf<R>();
    if (act[k] && s > R(0)) u[k] = min(u[k], -(lr[k] + c0[k]) / s);
  }
  // probe step from the previous roots
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    R w = uw[k];
    R t = lr[k] - w;
    R e = dd_ex2(-fabs(t) * L2E);
    R ie = dd_rcp(R(1) + e);
    R sp = max(t, R(0)) + dd_lg2(R(1) + e) * LN2;
    R sig = t >= R(0) ? ie : e * ie;
    R g = one_s * w + c0[k] + sp;
    R wn = w - g * dd_rcp(one_s - sig);
    if (act[k] && wn == wn && wn < u[k]) u[k] = wn;
  }
  for (int it = 0; it < maxit && (act[0] || act[1]); ++it) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      R t = lr[k] - u[k];
      R e = dd_ex2(-fabs(t) * L2E);
      R ie = dd_rcp(R(1) + e);
      R sp = max(t, R(0)) + dd_lg2(R(1) + e) * LN2;
      R sig = t >= R(0) ? ie : e * ie;
      R g = one_s * u[k] + c0[k] + sp;
      R du = g * dd_rcp(one_s - sig);
      if (act[k]) {
        u[k] -= du;
        if (fabs(du) <= tol * max(R(1), fabs(u[k]))) act[k] = false;
      }
    }
  }
}

// mu phi((p0 + d)/mu) - mu phi(p0/mu) with phi(s) = s log s - s + 1, written as
//   d (log(p0/mu) - 1) + (p0 + d) log1p(d/p0),
// an identity whose float evaluation errs by ~1e-7 |d| (both logarithms enter
// multiplied by the change), unlike the difference of the two terms (~1e-7 p0).
// log_mu: natural log of mu.  The result is returned in double for summation.
__device__ __forceinline__ double kl_change_f(double p0, double d, float log_mu) {
  const double p1 = p0 + d;
  if (p0 <= 0.0) {   // mu phi(0) = mu
    if (p1 <= 0.0) return 0.0;
    const float p1f = (float)p1;
    return (double)(p1f * (dd_lg2(p1f) * (float)DD_LN2 - log_mu - 1.0f));
  }
  const float p0f = (float)p0, df = (float)d;
  const float l0 = dd_lg2(p0f) * (float)DD_LN2 - log_mu;
  const float l1p = log1pf(df / p0f);
  if (p1 <= 0.0) return (double)(df * (l0 - 1.0f));   // limit p1 log(p1/p0) -> 0
  return (double)(df * (l0 - 1.0f)) + p1 * (double)l1p;
}

// v[k] for a run-time k in 0..3 without indexing a local array (keeps it in registers).
__device__ __forceinline__ double pick4(const double (&v)[4], int k) {
  return k == 0 ? v[0] : (k == 1 ? v[1] : (k == 2 ? v[2] : v[3]));
}

__device__ __forceinline__ double box_value(const BoxRec& b, const double* arena, int y1, int y2) {
  int a = y1 - b.k0, c = y2 - b.l0;
  if (a < 0 || c < 0 || a >= b.H || c >= b.W) return 0.0;
  return arena[b.off + (long long)a * b.W + c];
}

}  // namespace

// One composite cell on one CTA: cell `cd` at position `cidx` of a sub-batch
// of `nbatch` cells.
template <typename R>
__device__ __forceinline__ void cell_solve_body(const DevState& S, const CellDesc cd, int cidx, int nbatch,
                                                unsigned char* smem_raw) {
  namespace cg = cooperative_groups;
  double* red = reinterpret_cast<double*>(smem_raw);  // 32 * 16 doubles (block reductions)
  __shared__ BoxRec sbox[4];
  __shared__ int sgeo[8];
  CellOut* out = S.cout + cidx;
  const unsigned long long t_start = dd_global_ns();
  const double* __restrict__ arena = S.arena[*S.cur];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int gtid = tid, gthr = nthr;
  const int N = S.N, s = S.s;
  const int nx1 = cd.nx1, nx2 = cd.nx2, nx = nx1 * nx2;
  auto csync = [&]() { __syncthreads(); };

  // ---------------------------------------------------------------- B_J
  if (tid == 0) {
    int k0 = 1 << 30, l0 = 1 << 30, k1 = -1, l1 = -1, slot = -1;
    for (int q = 0; q < 4; ++q) {
      BoxRec b = {0, 0, 0, 0, 0};
      if (cd.mem[q] >= 0) b = S.box[cd.mem[q]];
      sbox[q] = b;
      if (cd.mem[q] < 0 || b.H * b.W == 0) continue;
      k0 = min(k0, b.k0); l0 = min(l0, b.l0);
      k1 = max(k1, b.k0 + b.H); l1 = max(l1, b.l0 + b.W);
    }
    int st = CELL_OK;
    if (k1 < 0) {
      st = CELL_EMPTY;
      k0 = l0 = k1 = l1 = 0;
    } else {
      k0 = max(0, k0 - S.margin); l0 = max(0, l0 - S.margin);
      k1 = min(N, k1 + S.margin); l1 = min(N, l1 + S.margin);
      int H = k1 - k0, W = l1 - l0;
      // boxes beyond the shared-memory capacity run from a global spill slot
      if (H * W > S.cap_ny || H > S.cap_side || W > S.cap_side) {
        int sl = S.spill_slots > 0 ? (int)atomicAdd(S.spill_count, 1u) : S.spill_slots;
        if (sl >= S.spill_slots) st = CELL_TOOBIG;
        else slot = sl;
      }
    }
    sgeo[0] = k0; sgeo[1] = l0; sgeo[2] = k1 - k0; sgeo[3] = l1 - l0;
    sgeo[4] = st; sgeo[7] = slot;
  }
  csync();
  const int k0 = sgeo[0], l0 = sgeo[1], H = sgeo[2], W = sgeo[3];
  if (sgeo[4] != CELL_OK) {
    if (tid == 0) {
      CellOut o;
      o.k0 = k0; o.l0 = l0; o.H = H; o.W = W; o.iters = 0; o.status = sgeo[4];
      o.D1 = o.D2 = 0; o.gap = 0.0; o.dKX[0] = o.dKX[1] = 0.0; o.slot = -1; o.usec = 0;
      for (int q = 0; q < 4; ++q) {
        int bi = cd.mem[q];
        o.Ct[q] = bi >= 0 ? S.Cc[bi] : 0.0;
        o.Ht[q] = bi >= 0 ? S.Hh[bi] : 0.0;
        o.mass[q] = 0.0;
      }
      *out = o;
      atomicOr(S.status, sgeo[4] == CELL_EMPTY ? ST_EMPTY : ST_TOOBIG);
    }
    return;
  }
  const int ny = H * W;

  // ------------------------------------------------------- shared layout
  // X-side arrays always live in shared memory; the Y-side arrays too unless
  // the box exceeds the shared capacity, then in the cell's spill slot
  // (global memory, L2-resident) sized for an N x N box.
  const int cap_nx = 4 * s * s;
  const int slot = sgeo[7];
  const bool spilled = slot >= 0;
  const int tsz = spilled ? 2 * s * N : 2 * s * S.cap_side;
  const int cap_ny = spilled ? N * N : S.cap_ny;
  R* xa = reinterpret_cast<R*>(smem_raw + 32 * 16 * sizeof(double));
  R* av = xa + cap_nx;
  R* g0 = av + cap_nx;
  R* Wv = g0 + cap_nx;
  R* lm = Wv + cap_nx;
  R* xa_nx = lm + cap_nx;    // next iterate of xa / a (double buffer of the X-update)
  R* av_nx = xa_nx + cap_nx;
  R* T = spilled ? reinterpret_cast<R*>(S.spill + (long long)slot * S.spill_stride) : av_nx + cap_nx;
  R* U = T + tsz;
  R* bl = U + tsz;
  R* lrho = bl + cap_ny;
  R* Zv = lrho + cap_ny;
  R* bv = Zv + cap_ny;
  R* lnu = bv + cap_ny;

  // ------------------------------------------------------- load Y side (a1)
  // rho = max(0, P_Y - nu_J)/nu and log nu on B_J; the same pass accumulates
  // the barycentre of nu_J, whose nearest pixel is the Y frame origin (so
  // that 2 q D.xi carries the cell's mean displacement).
  double a_tot = 0.0;   // |nu_{-J}| on B_J (translation step)
  {
    double m3[4] = {0.0, 0.0, 0.0, 0.0};
    for (int u = tid; u < ny; u += nthr) {
      int kk = u / W, ll = u - kk * W;
      int y1 = k0 + kk, y2 = l0 + ll, y = y1 * N + y2;
      double nuJ = 0.0;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) nuJ += box_value(sbox[q4], arena, y1, y2);
      double nuy = S.nu[y];
      const double num = fmax(0.0, S.PY[y] - nuJ);
      R rho = R(num) / R(nuy);
      lrho[u] = rho > R(0) ? dd_lg2(rho) * R(DD_LN2) : -dd_inf<R>();
      lnu[u] = R(S.lognu[y]);
      m3[0] += nuJ; m3[1] += nuJ * kk; m3[2] += nuJ * ll; m3[3] += num;
    }
    block_sum<4>(m3, red);
    a_tot = m3[3];
    if (tid == 0) {
      int c1 = H / 2, c2 = W / 2;
      if (m3[0] > 0.0) {
        c1 = min(H - 1, max(0, (int)lrint(m3[1] / m3[0])));
        c2 = min(W - 1, max(0, (int)lrint(m3[2] / m3[0])));
      }
      sgeo[5] = c1; sgeo[6] = c2;
    }
    __syncthreads();
  }
  const int xc1 = cd.i0 + nx1 / 2, xc2 = cd.j0 + nx2 / 2;
  const int yc1 = k0 + sgeo[5], yc2 = l0 + sgeo[6];
  const int D1 = xc1 - yc1, D2 = xc2 - yc2;
  const int offr = (k0 - cd.i0) + D1, offc = (l0 - cd.j0) + D2;
  const double eps = S.eps, lam = S.lam;
  const double q = S.h * S.h / eps;
  const double sl = eps / lam;            // s = eps/lam
  const double rr = lam / (eps + lam);    // r = lam/(eps+lam)
  const R q2 = R(q * DD_LOG2E), qR = R(q), sR = R(sl), rR = R(rr);

  // ------------------------------------------------------- load X side
  const double inv_eps = 1.0 / eps;
  double acc2[2] = {0.0, 0.0};
  for (int t = tid; t < nx; t += nthr) {
    int r = t / nx2, c = t - r * nx2;
    int x = (cd.i0 + r) * N + cd.j0 + c;
    int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
    acc2[0] += S.alpha[x] * inv_eps - 2.0 * q * (double)(D1 * xi1 + D2 * xi2);
    acc2[1] += S.mu[x];
  }
  block_sum<2>(acc2, red);
  double A = acc2[0] / nx;
  const double muJ = acc2[1];
  const double qD2 = q * (double)(D1 * D1 + D2 * D2);
  R sB = R(sl * (qD2 - A));   // s B with B = q|D|^2 - A
  const R cEta1 = R(sl * 2.0 * q * D1), cEta2 = R(sl * 2.0 * q * D2);
  R cA = R(-(1.0 - rr) * A);
  R gA = R(-sl * A);          // -s A: the A part of -alpha/lam
  const R cD1 = R(2.0 * (1.0 - rr) * q * D1), cD2 = R(2.0 * (1.0 - rr) * q * D2);
  for (int t = tid; t < nx; t += nthr) {
    int r = t / nx2, c = t - r * nx2;
    int x = (cd.i0 + r) * N + cd.j0 + c;
    int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
    double lin = 2.0 * q * (double)(D1 * xi1 + D2 * xi2);
    R a = R(S.alpha[x] * inv_eps - lin - A);
    R l = R(S.logmu[x]);
    av[t] = a;
    lm[t] = l;
    g0[t] = R(-sl * lin);
    xa[t] = (a + l) * R(DD_LOG2E);
  }
  csync();

  // ------------------------------------------------------- Sinkhorn loop
  // Barriers per iteration: after each of the five passes.  The X-update is
  // computed speculatively inside the last pass into the second buffer, and
  // the gap is reduced from per-warp partials after that pass's barrier.
  const double tol = S.err * muJ;
  const R LN2 = R(DD_LN2), L2E = R(DD_LOG2E);
  R* gpart = reinterpret_cast<R*>(red) + 32 * 12;   // per-warp gap partials
  R* apart = gpart + 32;                             // per-warp <e^{-alpha/lam}, mu> (translation step)
  R* bpart = gpart + 64;                             // per-warp <e^{-beta/lam}, nu>
  const bool ti = S.ti && sl > 0.0;
  const int lane = tid & 31, wid = tid >> 5, nwarp = nthr >> 5;
  int it = 0;
  double gap = 0.0;
  bool first = true;
  const bool fused_y = ny * 2 > gthr;   // large boxes: one lane per y, LSE and Newton fused
  R *xa_c = xa, *av_c = av;          // current iterate
  R *xa_n = xa_nx, *av_n = av_nx;    // next iterate
  for (;;) {
    ++it;
    // Y-half, pass over columns of X: T(r, ll) = log2 sum_c 2^{xa(r,c) - q2 (c - ll - offc)^2}
    {
      const int nt = nx1 * W, P = lanes_per_target(nt, nx2, gthr), ni = (nt * P + 31) & ~31;
      for (int i = gtid; i < ni; i += gthr) {
        const int tg0 = i / P, part = i - tg0 * P, tg = min(tg0, nt - 1);
        const int r = tg / W, ll = tg - r * W;
        const R* row = xa_c + r * nx2;
        R v = lse2_group<R>([&](int m) { return row[m]; }, nx2, R(ll + offc), q2, T[tg], !first, part, P);
        __syncwarp();
        if (part == 0 && tg0 < nt) T[tg] = v;
      }
    }
    csync();
    // Y-half, pass over rows of X: Z(kk, ll), then the Newton root per y (a3)
    R bsum = R(0);
    if (fused_y) {
      // every lane runs the same number of rounds (lse2_group is warp-collective)
      const int rounds = (ny + 2 * gthr - 1) / (2 * gthr);
      for (int rd = 0; rd < rounds; ++rd) {
        const int u = gtid + rd * 2 * gthr;
        const int uu[2] = {min(u, ny - 1), min(u + gthr, ny - 1)};
        const bool ok[2] = {u < ny, u + gthr < ny};
        R lr[2], c0[2], uw[2], root[2], Zn[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int kk = uu[k] / W, ll = uu[k] - kk * W;
          R Z2 = lse2_group<R>([&](int m) { return T[m * W + ll]; }, nx1, R(kk + offr), q2, Zv[uu[k]], !first, 0, 1);
          Zn[k] = Z2 * LN2;
          R eta1 = R(k0 + kk - yc1), eta2 = R(l0 + ll - yc2);
          c0[k] = sB - cEta1 * eta1 - cEta2 * eta2 - sR * Zn[k];
          lr[k] = lrho[uu[k]];
          uw[k] = first ? dd_inf<R>() : bv[uu[k]] + Zn[k];
        }
        newton_u2<R>(lr, c0, uw, sR, S.newton_maxit, root);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (!ok[k]) continue;
          Zv[uu[k]] = Zn[k] * L2E;
          R b = root[k] - Zn[k];
          bv[uu[k]] = b;
          bl[uu[k]] = (b + lnu[uu[k]]) * L2E;
          // nu e^{-beta/lam}: -s beta/eps = -(s root + c0)
          if (ti) bsum += dd_ex2((lnu[uu[k]] - sR * root[k] - c0[k]) * L2E);
        }
      }
    } else {
      const int P = lanes_per_target(ny, nx1, gthr), ni = (ny * P + 31) & ~31;
      for (int i = gtid; i < ni; i += gthr) {
        const int u0 = i / P, part = i - u0 * P, u = min(u0, ny - 1);
        const int kk = u / W, ll = u - kk * W;
        R Z2 = lse2_group<R>([&](int m) { return T[m * W + ll]; }, nx1, R(kk + offr), q2, Zv[u], !first, part, P);
        __syncwarp();
        if (part == 0 && u0 < ny) Zv[u] = Z2;
      }
      csync();
      for (int u = gtid; u < ny; u += 2 * gthr) {
        const int uu[2] = {u, min(u + gthr, ny - 1)};
        R lr[2], c0[2], uw[2], root[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int kk = uu[k] / W, ll = uu[k] - kk * W;
          R Zn = Zv[uu[k]] * LN2;
          R eta1 = R(k0 + kk - yc1), eta2 = R(l0 + ll - yc2);
          c0[k] = sB - cEta1 * eta1 - cEta2 * eta2 - sR * Zn;
          lr[k] = lrho[uu[k]];
          uw[k] = first ? dd_inf<R>() : bv[uu[k]] + Zn;
        }
        newton_u2<R>(lr, c0, uw, sR, S.newton_maxit, root);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k == 1 && u + gthr >= ny) break;
          R b = root[k] - Zv[uu[k]] * LN2;
          bv[uu[k]] = b;
          bl[uu[k]] = (b + lnu[uu[k]]) * L2E;
          if (ti) bsum += dd_ex2((lnu[uu[k]] - sR * root[k] - c0[k]) * L2E);
        }
      }
    }
    if (ti) {
      bsum = warp_sum(bsum);
      if (lane == 0) bpart[wid] = bsum;
    }
    csync();
    // X-half, pass over columns of B_J: U(kk, c) = log2 sum_ll 2^{bl(kk,ll) - q2 (ll - (c - offc))^2}
    {
      const int nt = H * nx2, P = lanes_per_target(nt, W, gthr), ni = (nt * P + 31) & ~31;
      for (int i = gtid; i < ni; i += gthr) {
        const int tg0 = i / P, part = i - tg0 * P, tg = min(tg0, nt - 1);
        const int kk = tg / nx2, c = tg - kk * nx2;
        const R* row = bl + kk * W;
        R v = lse2_group<R>([&](int m) { return row[m]; }, W, R(c - offc), q2, U[tg], !first, part, P);
        __syncwarp();
        if (part == 0 && tg0 < nt) U[tg] = v;
      }
    }
    csync();
    // X-half, pass over rows of B_J: W, the gap terms (a4) and the next a (a2)
    {
      R gl = R(0), asum = R(0);
      const int P = lanes_per_target(nx, H, gthr), ni = (nx * P + 31) & ~31;
      for (int i = gtid; i < ni; i += gthr) {
        const int tg0 = i / P, part = i - tg0 * P, t = min(tg0, nx - 1);
        const int r = t / nx2, c = t - r * nx2;
        R W2 = lse2_group<R>([&](int m) { return U[m * nx2 + c]; }, H, R(r - offr), q2, Wv[t], !first, part, P);
        __syncwarp();
        if (part == 0 && tg0 < nx) {
          Wv[t] = W2;
          R a = av_c[t];
          R tt = a + W2 * LN2;         // log(P_X pi / mu)
          R g = gA + g0[t] - sR * a;   // -alpha/lam
          gl += dd_ex2((lm[t] + g) * L2E) * dd_psi<R>(tt - g);
          R xi1 = R(cd.i0 + r - xc1), xi2 = R(cd.j0 + c - xc2);
          R an = cA - rR * W2 * LN2 - cD1 * xi1 - cD2 * xi2;
          av_n[t] = an;
          xa_n[t] = (an + lm[t]) * L2E;
          if (ti) asum += dd_ex2((lm[t] + gA + g0[t] - sR * an) * L2E);   // mu e^{-alpha_new/lam}
        }
      }
      gl = warp_sum(gl);
      if (lane == 0) gpart[wid] = gl;
      if (ti) {
        asum = warp_sum(asum);
        if (lane == 0) apart[wid] = asum;
      }
    }
    csync();
    {
      R gs = R(0);
      for (int w = 0; w < nwarp; ++w) gs += gpart[w];
      gap = (double)gs;
    }
    first = false;
    if ((S.err >= 0.0 && gap <= tol) || it >= S.maxit || !(gap == gap)) break;
    if (ti) {
      // translation step: alpha += t*, e^{t*/lam} = (a + sqrt(a^2 + 4 A_s B_s)) / (2 B_s); in the
      // cell frame alpha/eps = A + a(xi) + 2qD.xi it moves A by t*/eps = log(u)/s (same in
      // every thread: the partials are replicated)
      double As = 0.0, Bs = 0.0;
      for (int w = 0; w < nwarp; ++w) {
        As += (double)apart[w];
        Bs += (double)bpart[w];
      }
      const double uu = (a_tot + sqrt(a_tot * a_tot + 4.0 * As * Bs)) / (2.0 * Bs);
      if (uu > 0.0 && uu < INFINITY) {
        A += log(uu) / sl;
        sB = R(sl * (qD2 - A));
        cA = R(-(1.0 - rr) * A);
        gA = R(-sl * A);
      }
    }
    // accept the X-update: swap the buffers
    R* tp = av_c; av_c = av_n; av_n = tp;
    tp = xa_c; xa_c = xa_n; xa_n = tp;
  }
  const bool nonfinite = !(gap == gap);

  // ------------------------------------------------------- epilogue (a5)
  // alpha, P_X of the new plan and the KL_X change: first CTA only.  With
  // balancing (one CTA per cell) P_X and the KL_X change follow the balancing.
  const bool bal = S.balance;
  const double th_s = 1.0 / nbatch;
  double dk[2] = {0.0, 0.0};
  double mubar[4] = {0.0, 0.0, 0.0, 0.0};   // balancing: mu_bar(X_q), X-marginal after one more X-half
  {
    for (int t = tid; t < nx; t += nthr) {
      int r = t / nx2, c = t - r * nx2;
      int x = (cd.i0 + r) * N + cd.j0 + c;
      int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
      double a = (double)av_c[t];
      S.alphanew[x] = eps * (A + a + 2.0 * q * (double)(D1 * xi1 + D2 * xi2));
      if (bal) {
        // av_n holds the X-half of the final beta (computed before the loop stopped)
        const int qd = 2 * (r >= s) + (c >= s);
        const double mb = exp(((double)lm[t] + (double)gA + (double)g0[t] - sl * (double)av_n[t]));
#pragma unroll
        for (int k = 0; k < 4; ++k) mubar[k] += k == qd ? mb : 0.0;   // static indices (no local memory)
        continue;
      }
      double p1 = (double)dd_ex2((lm[t] + av_c[t]) * L2E + Wv[t]);
      S.PXnew[x] = p1;
      double p0 = S.PX[x];
      if (sizeof(R) == 8) {
        double m = S.mu[x];
        double ps = (1.0 - th_s) * p0 + th_s * p1;
        double k0v = dd_kl_term(p0, m);
        dk[0] += dd_kl_term(p1, m) - k0v;
        dk[1] += dd_kl_term(ps, m) - k0v;
      } else {
        // float cell solve: the KL_X changes from the cancellation-free form
        // (the error scales with the change p1 - p0, not with p)
        dk[0] += kl_change_f(p0, p1 - p0, lm[t]);
        dk[1] += kl_change_f(p0, th_s * (p1 - p0), lm[t]);
      }
    }
    if (bal) block_sum<4>(mubar, red);
    else block_sum<2>(dk, red);
  }

  R hs[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) hs[k] = R(0);
  const int nhr = nx1 > s ? 2 : 1, nhc = nx2 > s ? 2 : 1;
  int nst;
  double* nut;
  {
    CellOut tmp;
    tmp.slot = slot;
    nut = cell_nut(S, tmp, cidx, &nst);
  }
  R* Te = T;                 // epilogue scratch spans T, U, bl, lrho (and Zv for the widest boxes)
  R* Ma = T + nx1 * W;
  R* Md = Ma + nx1 * W;
  // Zv (the final Z) serves as the shift of the quadrant sums unless Md reaches it
  const bool zok = Md + nx1 * W <= Zv;
  for (int hc = 0; hc < nhc; ++hc) {
    const int cb = hc * s, ce = min(nx2, cb + s);
    // rows of X_J against columns of B_J, restricted to the column half hc
    for (int t = gtid; t < nx1 * W; t += gthr) {
      int r = t / W, ll = t - r * W;
      const R* row = xa_c + r * nx2;
      R ma, md;
      const R T2 = lse_moments<R>([&](int m) { return row[m]; }, [&](int m) { return av_c[r * nx2 + m]; },
                                  [&](int) { return R(0); }, qR, R(D2), cb, ce, R(ll + offc), q2, R(0), false, ma,
                                  md);
      Te[t] = T2;
      Ma[t] = ma;
      Md[t] = md;
    }
    csync();
    for (int u = gtid; u < ny; u += gthr) {
      int kk = u / W, ll = u - kk * W;
      int y = (k0 + kk) * N + l0 + ll;
      R ctr = R(kk + offr);
      double nuy = S.nu[y];
      // Z of the last iteration: the log-sum-exp over all rows of the full-row
      // T, an upper bound of every quadrant's sum at this y
      const R zsh = zok ? Zv[u] : R(0);
      for (int hr = 0; hr < nhr; ++hr) {
        const int rb = hr * s, re = min(nx1, rb + s);
        R ma, md;
        const R P2 = lse_moments<R>(
            [&](int m) { return Te[m * W + ll]; }, [&](int m) { return Ma[m * W + ll]; },
            [&](int m) { return Md[m * W + ll]; }, qR, R(D1), rb, re, ctr, q2, zsh, zok, ma, md);
        const int qd = 2 * hr + hc;
        R nt = R(nuy) * dd_ex2(bv[u] * L2E + P2);
        nut[qd * nst + u] = (double)nt;
        hs[qd] += nt * (ma + bv[u]);
        hs[4 + qd] += nt * md;
        hs[8 + qd] += nt;
      }
    }
    __threadfence();
    csync();
  }
  if (bal) {
    // ---- balancing (Section 5.3, Eq. balancing): targets m_q = mu_bar(X_q) |nu_J| / mu_bar(X_J);
    // donors scale their rows by m_q/|nu_q|, receivers by 1 + D(y) w_q / nu_q(y) with the donated
    // field D(y) = sum_d (|nu_d| - m_d) nu_d(y)/|nu_d| and w_q = deficit_q / total excess.
    double ms[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ms[k] = (double)hs[8 + k];
    block_sum<4>(ms, red);
    double mJ = 0.0, mbJ = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) { mJ += ms[k]; mbJ += mubar[k]; }
    double fd[4], rd[4], wr[4];   // donor factor, donor weight in D, receiver share
    double Ex = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double mk = mbJ > 0.0 ? mubar[k] * mJ / mbJ : 0.0;
      const double e = ms[k] - mk;
      fd[k] = 1.0; rd[k] = 0.0; wr[k] = 0.0;
      if (e > 0.0 && ms[k] > 0.0) { fd[k] = mk / ms[k]; rd[k] = e / ms[k]; Ex += e; }
      else if (e < 0.0) wr[k] = -e;
    }
    const bool move = Ex > 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) wr[k] = move ? wr[k] / Ex : 0.0;
    // rho_q(u) from the unbalanced marginals in nut
    auto rho_at = [&](int u, double (&rho)[4]) {
      double nv[4], D = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int hr = k >> 1, hc = k & 1;
        nv[k] = (hr < nhr && hc < nhc) ? nut[k * nst + u] : 0.0;
        D += rd[k] * nv[k];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        rho[k] = fd[k];
        if (wr[k] > 0.0 && nv[k] > 0.0) rho[k] = 1.0 + D * wr[k] / nv[k];
      }
    };
    // pass B: C and H of the balanced plan from the same per-y sums, weighted by rho
    if (move) {
#pragma unroll
      for (int k = 0; k < 12; ++k) hs[k] = R(0);
      for (int hc = 0; hc < nhc; ++hc) {
        const int cb = hc * s, ce = min(nx2, cb + s);
        for (int t = tid; t < nx1 * W; t += nthr) {
          int r = t / W, ll = t - r * W;
          const R* row = xa_c + r * nx2;
          R ctr = R(ll + offc);
          R T2 = lse2_1d<R>([&](int m) { return row[cb + m]; }, ce - cb, ctr - R(cb), q2, R(0), false);
          R sw = 0, sa = 0, sd = 0;
          for (int c = cb; c < ce; ++c) {
            R d = R(c) - ctr;
            R w = dd_ex2(row[c] - q2 * d * d - T2);
            sw += w;
            sa += w * (av_c[r * nx2 + c] - qR * d * d);
            R dt = d + R(D2);
            sd += w * dt * dt;
          }
          R isw = R(1) / sw;
          Te[t] = T2;
          Ma[t] = sa * isw;
          Md[t] = sd * isw;
        }
        __syncthreads();
        for (int u = tid; u < ny; u += nthr) {
          int kk = u / W, ll = u - kk * W;
          R ctr = R(kk + offr);
          double rho[4];
          rho_at(u, rho);
          for (int hr = 0; hr < nhr; ++hr) {
            const int rb = hr * s, re = min(nx1, rb + s);
            R P2 = lse2_1d<R>([&](int m) { return Te[(rb + m) * W + ll]; }, re - rb, ctr - R(rb), q2, R(0), false);
            R sw = 0, sa = 0, sd = 0;
            for (int r = rb; r < re; ++r) {
              R d = R(r) - ctr;
              R w = dd_ex2(Te[r * W + ll] - q2 * d * d - P2);
              sw += w;
              sa += w * (Ma[r * W + ll] - qR * d * d);
              R dt = d + R(D1);
              sd += w * (dt * dt + Md[r * W + ll]);
            }
            R isw = R(1) / sw;
            const int qd = 2 * hr + hc;
            const double nt = nut[qd * nst + u];
            const double rh = pick4(rho, qd);
            const double nh = rh * nt;
            hs[qd] += R(nh * ((double)(sa * isw) + (double)bv[u] + (rh > 0.0 ? log(rh) : 0.0)));
            hs[4 + qd] += R(nh * (double)(sd * isw));
            hs[8 + qd] += R(nh);
          }
        }
        __syncthreads();
      }
    }   // nothing moves: the sums of pass A stand
    // P_X of the balanced plan: per quadrant, one more X-pass with log2 rho_q added to b + log nu
    R* Lq = bl;
    for (int qd = 0; qd < 4; ++qd) {
      const int hr = qd >> 1, hc = qd & 1;
      if (hr >= nhr || hc >= nhc) continue;
      const int cb = hc * s, ce = min(nx2, cb + s), rb = hr * s, re = min(nx1, rb + s);
      for (int u = tid; u < ny; u += nthr) {
        double rho[4];
        rho_at(u, rho);
        const double rq = pick4(rho, qd);
        const double lr = rq > 0.0 ? log2(rq) : -INFINITY;
        Lq[u] = R(((double)bv[u] + (double)lnu[u]) * DD_LOG2E + lr);
      }
      __syncthreads();
      for (int t = tid; t < H * (ce - cb); t += nthr) {
        const int kk = t / (ce - cb), c = cb + (t - kk * (ce - cb));
        U[kk * nx2 + c] = lse2_1d<R>([&](int m) { return Lq[kk * W + m]; }, W, R(c - offc), q2, R(0), false);
      }
      __syncthreads();
      for (int t = tid; t < (re - rb) * (ce - cb); t += nthr) {
        const int r = rb + t / (ce - cb), c = cb + (t - (t / (ce - cb)) * (ce - cb));
        const int tx = r * nx2 + c;
        R W2 = lse2_1d<R>([&](int m) { return U[m * nx2 + c]; }, H, R(r - offr), q2, R(0), false);
        const int x = (cd.i0 + r) * N + cd.j0 + c;
        double p1 = (double)dd_ex2((lm[tx] + av_c[tx]) * L2E + W2);
        if (!move) p1 = (double)dd_ex2((lm[tx] + av_c[tx]) * L2E + Wv[tx]);
        S.PXnew[x] = p1;
        double p0 = S.PX[x], m = S.mu[x];
        double ps = (1.0 - th_s) * p0 + th_s * p1;
        double k0v = dd_kl_term(p0, m);
        dk[0] += dd_kl_term(p1, m) - k0v;
        dk[1] += dd_kl_term(ps, m) - k0v;
      }
      __syncthreads();
    }
    block_sum<2>(dk, red);
    // the balanced marginals
    if (move) {
      for (int u = tid; u < ny; u += nthr) {
        double rho[4];
        rho_at(u, rho);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if ((k >> 1) < nhr && (k & 1) < nhc) nut[k * nst + u] *= rho[k];
      }
    }
    __threadfence();
    __syncthreads();
  }
  // change of P_Y pi for the step-size decision
  for (int u = gtid; u < ny; u += gthr) {
    int kk = u / W, ll = u - kk * W;
    int y1 = k0 + kk, y2 = l0 + ll;
    double dlt = 0.0;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      if (cd.mem[q4] < 0) continue;
      int hr = q4 >> 1, hc = q4 & 1;
      if (hr >= nhr || hc >= nhc) continue;
      dlt += nut[q4 * nst + u] - box_value(sbox[q4], arena, y1, y2);
    }
    if (dlt != 0.0) atomicAdd(S.dPY + y1 * N + y2, dlt);
  }
  double hsd[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) hsd[k] = (double)hs[k];
  block_sum<12>(hsd, red);
  if (tid == 0) {
    CellOut o;
    o.k0 = k0; o.l0 = l0; o.H = H; o.W = W;
    o.iters = it;
    o.status = nonfinite ? CELL_NONFINITE : ((S.err >= 0.0 && gap > tol) ? CELL_MAXIT : CELL_OK);
    o.D1 = D1; o.D2 = D2;
    o.slot = slot;
    o.usec = (int)min((dd_global_ns() - t_start) / 1000ull, 2147483647ull);
    o.gap = gap;
    o.dKX[0] = dk[0]; o.dKX[1] = dk[1];
    for (int q4 = 0; q4 < 4; ++q4) {
      int bi = cd.mem[q4];
      o.Ct[q4] = S.h * S.h * hsd[4 + q4];
      o.mass[q4] = hsd[8 + q4];
      o.Ht[q4] = bi >= 0 ? hsd[q4] - hsd[8 + q4] + S.muinu[bi] : 0.0;
    }
    *out = o;   // the decision kernel adds the sub-batch's counters
    if (nonfinite) atomicOr(S.status, ST_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// One cell solved by a cluster of C <= S.dist_c CTAs (the layout's capacities
// were sized for S.dist_c, a smaller C only leaves more room), split by rows
// of its Y box.
// CTA r owns rows [kb, ke) of B_J: the Y-side arrays (log rho, log nu, Z, beta,
// beta + log nu) of those rows live in its shared memory only, so a cluster
// holds C times the Y points of one CTA and the largest cells of a sub-batch
// spread over C SMs.  Per iteration:
//   T pass  (rows of X against the columns of B_J, the same for every slab):
//           targets split over the cluster, every result written to all CTAs
//           (distributed shared memory); cluster barrier;
//   Z pass and the Newton roots of the Y-half on the own rows;
//   U pass (rows of B_J against the columns of X) on the own rows;
//   W partial: the column log-sum-exp of the X-half over the own rows only,
//           written to the exchange buffer of every CTA; cluster barrier;
//   every CTA combines the C partials of each x in rank order (so all CTAs
//           hold the same W, gap and next alpha) -- no further exchange.
// The epilogue splits the rows-of-X pass the same way and sums the
// per-quadrant terms of the own rows; the first CTA adds the cluster's sums.
constexpr int kDistMaxC = 8;

template <typename R>
__device__ __forceinline__ void cell_solve_dist(const DevState& S, const CellDesc cd, int cidx, int nbatch,
                                                int crank, int C, unsigned char* smem_raw) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  double* red = reinterpret_cast<double*>(smem_raw);   // 32 * 16 doubles (block reductions)
  __shared__ BoxRec dbox[4];
  __shared__ int dgeo[8];
  __shared__ double dx[kDistMaxC * 16];                 // partial sums of every CTA of the cluster
  CellOut* out = S.cout + cidx;
  const unsigned long long t_start = dd_global_ns();
  const double* __restrict__ arena = S.arena[*S.cur];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int gtid = crank * nthr + tid, gthr = C * nthr;
  const int N = S.N, s = S.s;
  const int nx1 = cd.nx1, nx2 = cd.nx2, nx = nx1 * nx2;
  auto csync = [&]() { cl.sync(); };

  // ---------------------------------------------------------------- B_J
  // every CTA computes the same box; the first one takes a spill slot for the
  // new marginals when the box exceeds the per-cell marginal buffer and tells
  // the others (its status decides for the whole cluster)
  if (tid == 0) {
    int k0 = 1 << 30, l0 = 1 << 30, k1 = -1, l1 = -1;
    for (int q = 0; q < 4; ++q) {
      BoxRec b = {0, 0, 0, 0, 0};
      if (cd.mem[q] >= 0) b = S.box[cd.mem[q]];
      dbox[q] = b;
      if (cd.mem[q] < 0 || b.H * b.W == 0) continue;
      k0 = min(k0, b.k0); l0 = min(l0, b.l0);
      k1 = max(k1, b.k0 + b.H); l1 = max(l1, b.l0 + b.W);
    }
    int st = CELL_OK;
    if (k1 < 0) {
      st = CELL_EMPTY;
      k0 = l0 = k1 = l1 = 0;
    } else {
      k0 = max(0, k0 - S.margin); l0 = max(0, l0 - S.margin);
      k1 = min(N, k1 + S.margin); l1 = min(N, l1 + S.margin);
    }
    const int H = k1 - k0, W = l1 - l0;
    dgeo[0] = k0; dgeo[1] = l0; dgeo[2] = H; dgeo[3] = W;
    if (crank == 0) {
      int slot = -1;
      const int hl = (H + C - 1) / C;
      if (st == CELL_OK && (H < C || W > S.dist_cap_w || hl > S.dist_cap_hl || hl * W > S.dist_cap_nyl))
        st = CELL_TOOBIG;   // excluded by k_cell_order; kept as a guard
      if (st == CELL_OK && H * W > S.cap_nut) {
        const int sl = S.spill_slots > 0 ? (int)atomicAdd(S.spill_count, 1u) : S.spill_slots;
        if (sl >= S.spill_slots) st = CELL_TOOBIG;
        else slot = sl;
      }
      for (int r = 0; r < C; ++r) {
        int* g = cl.map_shared_rank(dgeo, r);
        g[4] = st;
        g[7] = slot;
      }
    }
  }
  csync();
  const int k0 = dgeo[0], l0 = dgeo[1], H = dgeo[2], W = dgeo[3];
  const int slot = dgeo[7];
  if (dgeo[4] != CELL_OK) {
    if (tid == 0 && crank == 0) {
      CellOut o;
      o.k0 = k0; o.l0 = l0; o.H = H; o.W = W; o.iters = 0; o.status = dgeo[4];
      o.D1 = o.D2 = 0; o.gap = 0.0; o.dKX[0] = o.dKX[1] = 0.0; o.slot = -1; o.usec = 0;
      for (int q = 0; q < 4; ++q) {
        const int bi = cd.mem[q];
        o.Ct[q] = bi >= 0 ? S.Cc[bi] : 0.0;
        o.Ht[q] = bi >= 0 ? S.Hh[bi] : 0.0;
        o.mass[q] = 0.0;
      }
      *out = o;
      atomicOr(S.status, dgeo[4] == CELL_EMPTY ? ST_EMPTY : ST_TOOBIG);
    }
    return;
  }
  const int kb = (int)(((long long)H * crank) / C), ke = (int)(((long long)H * (crank + 1)) / C);
  const int Hl = ke - kb, nyl = Hl * W;

  // ------------------------------------------------------- shared layout
  const int cap_nx = 4 * s * s;
  R* xa = reinterpret_cast<R*>(smem_raw + 32 * 16 * sizeof(double));
  R* av = xa + cap_nx;
  R* g0 = av + cap_nx;
  R* Wv = g0 + cap_nx;       // W of the X-half, combined over the cluster
  R* lm = Wv + cap_nx;
  R* xa_nx = lm + cap_nx;
  R* av_nx = xa_nx + cap_nx;
  R* Wp = av_nx + cap_nx;    // own rows' part of W (the shift of the next iteration)
  R* Wx = Wp + cap_nx;       // C x cap_nx: the parts of all CTAs
  R* T = Wx + C * cap_nx;    // nx1 x W
  R* U = T + 2 * s * S.dist_cap_w;   // Hl x nx2
  R* bl = U + 2 * s * S.dist_cap_hl;
  R* lrho = bl + S.dist_cap_nyl;
  R* Zv = lrho + S.dist_cap_nyl;
  R* bv = Zv + S.dist_cap_nyl;
  R* lnu = bv + S.dist_cap_nyl;

  // ------------------------------------------------- load Y side (a1), own rows
  // rho = max(0, P_Y - nu_J)/nu and log nu; the barycentre of nu_J (the Y frame
  // origin) is summed over the whole box from every CTA's part
  int c1, c2;
  {
    double m3[3] = {0.0, 0.0, 0.0};
    for (int ul = tid; ul < nyl; ul += nthr) {
      const int kl = ul / W, ll = ul - kl * W, kk = kb + kl;
      const int y1 = k0 + kk, y2 = l0 + ll, y = y1 * N + y2;
      double nuJ = 0.0;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) nuJ += box_value(dbox[q4], arena, y1, y2);
      const double num = fmax(0.0, S.PY[y] - nuJ);
      const R rho = R(num) / R(S.nu[y]);
      lrho[ul] = rho > R(0) ? dd_lg2(rho) * R(DD_LN2) : -dd_inf<R>();
      lnu[ul] = R(S.lognu[y]);
      m3[0] += nuJ; m3[1] += nuJ * kk; m3[2] += nuJ * ll;
    }
    block_sum<3>(m3, red);
    if (tid == 0)
      for (int r = 0; r < C; ++r) {
        double* px = cl.map_shared_rank(dx, r);
        for (int k = 0; k < 3; ++k) px[crank * 16 + k] = m3[k];
      }
    csync();
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int r = 0; r < C; ++r) { t0 += dx[r * 16]; t1 += dx[r * 16 + 1]; t2 += dx[r * 16 + 2]; }
    c1 = H / 2; c2 = W / 2;
    if (t0 > 0.0) {
      c1 = min(H - 1, max(0, (int)lrint(t1 / t0)));
      c2 = min(W - 1, max(0, (int)lrint(t2 / t0)));
    }
  }
  const int xc1 = cd.i0 + nx1 / 2, xc2 = cd.j0 + nx2 / 2;
  const int yc1 = k0 + c1, yc2 = l0 + c2;
  const int D1 = xc1 - yc1, D2 = xc2 - yc2;
  const int offr = (k0 - cd.i0) + D1, offc = (l0 - cd.j0) + D2;
  const double eps = S.eps, lam = S.lam;
  const double q = S.h * S.h / eps;
  const double sl = eps / lam;
  const double rr = lam / (eps + lam);
  const R q2 = R(q * DD_LOG2E), qR = R(q), sR = R(sl), rR = R(rr);

  // ------------------------------------------------------- load X side (every CTA)
  const double inv_eps = 1.0 / eps;
  double acc2[2] = {0.0, 0.0};
  for (int t = tid; t < nx; t += nthr) {
    const int r = t / nx2, c = t - r * nx2;
    const int x = (cd.i0 + r) * N + cd.j0 + c;
    const int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
    acc2[0] += S.alpha[x] * inv_eps - 2.0 * q * (double)(D1 * xi1 + D2 * xi2);
    acc2[1] += S.mu[x];
  }
  block_sum<2>(acc2, red);
  const double A = acc2[0] / nx;
  const double muJ = acc2[1];
  const double qD2 = q * (double)(D1 * D1 + D2 * D2);
  const R sB = R(sl * (qD2 - A));
  const R cEta1 = R(sl * 2.0 * q * D1), cEta2 = R(sl * 2.0 * q * D2);
  const R cA = R(-(1.0 - rr) * A);
  const R gA = R(-sl * A);
  const R cD1 = R(2.0 * (1.0 - rr) * q * D1), cD2 = R(2.0 * (1.0 - rr) * q * D2);
  for (int t = tid; t < nx; t += nthr) {
    const int r = t / nx2, c = t - r * nx2;
    const int x = (cd.i0 + r) * N + cd.j0 + c;
    const int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
    const double lin = 2.0 * q * (double)(D1 * xi1 + D2 * xi2);
    const R a = R(S.alpha[x] * inv_eps - lin - A);
    const R l = R(S.logmu[x]);
    av[t] = a;
    lm[t] = l;
    g0[t] = R(-sl * lin);
    xa[t] = (a + l) * R(DD_LOG2E);
  }
  __syncthreads();

  // ------------------------------------------------------- Sinkhorn loop
  const double tol = S.err * muJ;
  const R LN2 = R(DD_LN2), L2E = R(DD_LOG2E);
  int it = 0;
  double gap = 0.0;
  bool first = true;
  R *xa_c = xa, *av_c = av, *xa_n = xa_nx, *av_n = av_nx;
  for (;;) {
    ++it;
    // Y-half, T(r, ll) = log2 sum_c 2^{xa(r,c) - q2 (c - ll - offc)^2}: split, to every CTA
    {
      const int nt = nx1 * W, P = lanes_per_target(nt, nx2, gthr), ni = (nt * P + 31) & ~31;
      for (int i = gtid; i < ni; i += gthr) {
        const int tg0 = i / P, part = i - tg0 * P, tg = min(tg0, nt - 1);
        const int r = tg / W, ll = tg - r * W;
        const R* row = xa_c + r * nx2;
        const R v = lse2_group<R>([&](int m) { return row[m]; }, nx2, R(ll + offc), q2, T[tg], !first, part, P);
        __syncwarp();
        if (part == 0 && tg0 < nt)
          for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(T + tg, rk) = v;
      }
    }
    csync();
    // Y-half on the own rows: Z(kk, ll) = log2 sum_r 2^{T(r,ll) - q2 (r - kk - offr)^2}, Newton (a3)
    if (nyl * 2 > nthr) {
      const int rounds = (nyl + 2 * nthr - 1) / (2 * nthr);
      for (int rd = 0; rd < rounds; ++rd) {
        const int u = tid + rd * 2 * nthr;
        const int uu[2] = {min(u, nyl - 1), min(u + nthr, nyl - 1)};
        const bool ok[2] = {u < nyl, u + nthr < nyl};
        R lr[2], c0[2], uw[2], root[2], Zn[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int kl = uu[k] / W, ll = uu[k] - kl * W, kk = kb + kl;
          const R Z2 =
              lse2_group<R>([&](int m) { return T[m * W + ll]; }, nx1, R(kk + offr), q2, Zv[uu[k]], !first, 0, 1);
          Zn[k] = Z2 * LN2;
          const R eta1 = R(k0 + kk - yc1), eta2 = R(l0 + ll - yc2);
          c0[k] = sB - cEta1 * eta1 - cEta2 * eta2 - sR * Zn[k];
          lr[k] = lrho[uu[k]];
          uw[k] = first ? dd_inf<R>() : bv[uu[k]] + Zn[k];
        }
        newton_u2<R>(lr, c0, uw, sR, S.newton_maxit, root);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (!ok[k]) continue;
          Zv[uu[k]] = Zn[k] * L2E;
          const R b = root[k] - Zn[k];
          bv[uu[k]] = b;
          bl[uu[k]] = (b + lnu[uu[k]]) * L2E;
        }
      }
    } else {
      const int P = lanes_per_target(nyl, nx1, nthr), ni = (nyl * P + 31) & ~31;
      for (int i = tid; i < ni; i += nthr) {
        const int u0 = i / P, part = i - u0 * P, u = min(u0, nyl - 1);
        const int kl = u / W, ll = u - kl * W, kk = kb + kl;
        const R Z2 = lse2_group<R>([&](int m) { return T[m * W + ll]; }, nx1, R(kk + offr), q2, Zv[u], !first,
                                   part, P);
        __syncwarp();
        if (part == 0 && u0 < nyl) Zv[u] = Z2;
      }
      __syncthreads();
      for (int u = tid; u < nyl; u += 2 * nthr) {
        const int uu[2] = {u, min(u + nthr, nyl - 1)};
        R lr[2], c0[2], uw[2], root[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int kl = uu[k] / W, ll = uu[k] - kl * W, kk = kb + kl;
          const R Zn = Zv[uu[k]] * LN2;
          const R eta1 = R(k0 + kk - yc1), eta2 = R(l0 + ll - yc2);
          c0[k] = sB - cEta1 * eta1 - cEta2 * eta2 - sR * Zn;
          lr[k] = lrho[uu[k]];
          uw[k] = first ? dd_inf<R>() : bv[uu[k]] + Zn;
        }
        newton_u2<R>(lr, c0, uw, sR, S.newton_maxit, root);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k == 1 && u + nthr >= nyl) break;
          const R b = root[k] - Zv[uu[k]] * LN2;
          bv[uu[k]] = b;
          bl[uu[k]] = (b + lnu[uu[k]]) * L2E;
        }
      }
    }
    __syncthreads();
    // X-half on the own rows: U(kl, c) = log2 sum_ll 2^{bl(kl,ll) - q2 (ll - (c - offc))^2}
    {
      const int nt = Hl * nx2, P = lanes_per_target(nt, W, nthr), ni = (nt * P + 31) & ~31;
      for (int i = tid; i < ni; i += nthr) {
        const int tg0 = i / P, part = i - tg0 * P, tg = min(tg0, nt - 1);
        const int kl = tg / nx2, c = tg - kl * nx2;
        const R* row = bl + kl * W;
        const R v = lse2_group<R>([&](int m) { return row[m]; }, W, R(c - offc), q2, U[tg], !first, part, P);
        __syncwarp();
        if (part == 0 && tg0 < nt) U[tg] = v;
      }
    }
    __syncthreads();
    // the own rows' part of W(r, c) = log2 sum_kk 2^{U(kk,c) - q2 (kk - (r - offr))^2}, to every CTA
    if (Hl > 0) {
      const int P = lanes_per_target(nx, Hl, nthr), ni = (nx * P + 31) & ~31;
      for (int i = tid; i < ni; i += nthr) {
        const int tg0 = i / P, part = i - tg0 * P, t = min(tg0, nx - 1);
        const int r = t / nx2, c = t - r * nx2;
        const R v = lse2_group<R>([&](int m) { return U[m * nx2 + c]; }, Hl, R(r - offr - kb), q2, Wp[t], !first,
                                  part, P);
        __syncwarp();
        if (part == 0 && tg0 < nx) {
          Wp[t] = v;
          for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(Wx + crank * cap_nx + t, rk) = v;
        }
      }
    } else {
      for (int t = tid; t < nx; t += nthr)
        for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(Wx + crank * cap_nx + t, rk) = -dd_inf<R>();
    }
    csync();
    // combine the parts (rank order: every CTA gets the same W), gap terms (a4), next alpha (a2)
    double gl = 0.0;
    for (int t = tid; t < nx; t += nthr) {
      R mx = -dd_inf<R>();
      for (int rk = 0; rk < C; ++rk) mx = max(mx, Wx[rk * cap_nx + t]);
      R W2 = mx;
      if (mx > -dd_inf<R>()) {
        R acc = R(0);
        for (int rk = 0; rk < C; ++rk) acc += dd_ex2(Wx[rk * cap_nx + t] - mx);
        W2 = mx + dd_lg2(acc);
      }
      Wv[t] = W2;
      const int r = t / nx2, c = t - r * nx2;
      const R a = av_c[t];
      const R tt = a + W2 * LN2;         // log(P_X pi / mu)
      const R g = gA + g0[t] - sR * a;   // -alpha/lam
      gl += (double)(dd_ex2((lm[t] + g) * L2E) * dd_psi<R>(tt - g));
      const R xi1 = R(cd.i0 + r - xc1), xi2 = R(cd.j0 + c - xc2);
      const R an = cA - rR * W2 * LN2 - cD1 * xi1 - cD2 * xi2;
      av_n[t] = an;
      xa_n[t] = (an + lm[t]) * L2E;
    }
    {
      double gv[1] = {gl};
      block_sum<1>(gv, red);
      gap = gv[0];
    }
    first = false;
    if ((S.err >= 0.0 && gap <= tol) || it >= S.maxit || !(gap == gap)) break;
    R* tp = av_c; av_c = av_n; av_n = tp;
    tp = xa_c; xa_c = xa_n; xa_n = tp;
  }
  const bool nonfinite = !(gap == gap);

  // ------------------------------------------------------- epilogue (a5)
  const double th_s = 1.0 / nbatch;
  double dk[2] = {0.0, 0.0};
  if (crank == 0) {
    for (int t = tid; t < nx; t += nthr) {
      const int r = t / nx2, c = t - r * nx2;
      const int x = (cd.i0 + r) * N + cd.j0 + c;
      const int xi1 = cd.i0 + r - xc1, xi2 = cd.j0 + c - xc2;
      S.alphanew[x] = eps * (A + (double)av_c[t] + 2.0 * q * (double)(D1 * xi1 + D2 * xi2));
      const double p1 = (double)dd_ex2((lm[t] + av_c[t]) * L2E + Wv[t]);
      S.PXnew[x] = p1;
      const double p0 = S.PX[x];
      if (sizeof(R) == 8) {
        const double m = S.mu[x];
        const double ps = (1.0 - th_s) * p0 + th_s * p1;
        const double k0v = dd_kl_term(p0, m);
        dk[0] += dd_kl_term(p1, m) - k0v;
        dk[1] += dd_kl_term(ps, m) - k0v;
      } else {
        dk[0] += kl_change_f(p0, p1 - p0, lm[t]);
        dk[1] += kl_change_f(p0, th_s * (p1 - p0), lm[t]);
      }
    }
    block_sum<2>(dk, red);
  }
  R hs[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) hs[k] = R(0);
  const int nhr = nx1 > s ? 2 : 1, nhc = nx2 > s ? 2 : 1;
  int nst;
  double* nut;
  {
    CellOut tmp;
    tmp.slot = slot;
    nut = cell_nut(S, tmp, cidx, &nst);
  }
  // rows of X against the columns of B_J per column half (split, to every CTA);
  // the region T .. Zv is free after the loop
  R* Te = T;
  R* Ma = T + nx1 * W;
  R* Md = Ma + nx1 * W;
  const bool zok = Md + nx1 * W <= Zv;   // Zv (the final Z, own rows) is intact: the quadrant sums' shift
  for (int hc = 0; hc < nhc; ++hc) {
    const int cb = hc * s, ce = min(nx2, cb + s);
    for (int t = gtid; t < nx1 * W; t += gthr) {
      const int r = t / W, ll = t - r * W;
      const R* row = xa_c + r * nx2;
      R ma, md;
      const R T2 = lse_moments<R>([&](int m) { return row[m]; }, [&](int m) { return av_c[r * nx2 + m]; },
                                  [&](int) { return R(0); }, qR, R(D2), cb, ce, R(ll + offc), q2, R(0), false, ma,
                                  md);
      for (int rk = 0; rk < C; ++rk) {
        *cl.map_shared_rank(Te + t, rk) = T2;
        *cl.map_shared_rank(Ma + t, rk) = ma;
        *cl.map_shared_rank(Md + t, rk) = md;
      }
    }
    csync();
    for (int ul = tid; ul < nyl; ul += nthr) {
      const int kl = ul / W, ll = ul - kl * W, kk = kb + kl;
      const int u = kk * W + ll;
      const int y = (k0 + kk) * N + l0 + ll;
      const R ctr = R(kk + offr);
      const double nuy = S.nu[y];
      const R zsh = zok ? Zv[ul] : R(0);   // the final Z: an upper bound of every quadrant's sum
      for (int hr = 0; hr < nhr; ++hr) {
        const int rb = hr * s, re = min(nx1, rb + s);
        R ma, md;
        const R P2 = lse_moments<R>(
            [&](int m) { return Te[m * W + ll]; }, [&](int m) { return Ma[m * W + ll]; },
            [&](int m) { return Md[m * W + ll]; }, qR, R(D1), rb, re, ctr, q2, zsh, zok, ma, md);
        const int qd = 2 * hr + hc;
        const R ntv = R(nuy) * dd_ex2(bv[ul] * L2E + P2);
        nut[qd * nst + u] = (double)ntv;
        hs[qd] += ntv * (ma + bv[ul]);
        hs[4 + qd] += ntv * md;
        hs[8 + qd] += ntv;
      }
    }
    csync();   // Te/Ma/Md are rewritten by the next column half
  }
  // change of P_Y pi for the step-size decision (own rows)
  for (int ul = tid; ul < nyl; ul += nthr) {
    const int kl = ul / W, ll = ul - kl * W, kk = kb + kl;
    const int u = kk * W + ll;
    const int y1 = k0 + kk, y2 = l0 + ll;
    double dlt = 0.0;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      if (cd.mem[q4] < 0) continue;
      const int hr = q4 >> 1, hc = q4 & 1;
      if (hr >= nhr || hc >= nhc) continue;
      dlt += nut[q4 * nst + u] - box_value(dbox[q4], arena, y1, y2);
    }
    if (dlt != 0.0) atomicAdd(S.dPY + y1 * N + y2, dlt);
  }
  double hsd[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) hsd[k] = (double)hs[k];
  block_sum<12>(hsd, red);
  if (tid == 0) {
    double* p0 = cl.map_shared_rank(dx, 0);
    for (int k = 0; k < 12; ++k) p0[crank * 16 + k] = hsd[k];
  }
  csync();
  if (crank != 0 || tid != 0) return;
  for (int k = 0; k < 12; ++k) {
    double a = 0.0;
    for (int r = 0; r < C; ++r) a += dx[r * 16 + k];
    hsd[k] = a;
  }
  CellOut o;
  o.k0 = k0; o.l0 = l0; o.H = H; o.W = W;
  o.iters = it;
  o.status = nonfinite ? CELL_NONFINITE : ((S.err >= 0.0 && gap > tol) ? CELL_MAXIT : CELL_OK);
  o.D1 = D1; o.D2 = D2;
  o.slot = slot;
  o.usec = (int)min((dd_global_ns() - t_start) / 1000ull, 2147483647ull);
  o.gap = gap;
  o.dKX[0] = dk[0]; o.dKX[1] = dk[1];
  for (int q4 = 0; q4 < 4; ++q4) {
    const int bi = cd.mem[q4];
    o.Ct[q4] = S.h * S.h * hsd[4 + q4];
    o.mass[q4] = hsd[8 + q4];
    o.Ht[q4] = bi >= 0 ? hsd[q4] - hsd[8 + q4] + S.muinu[bi] : 0.0;
  }
  *out = o;   // the decision kernel adds the sub-batch's counters
  if (nonfinite) atomicOr(S.status, ST_NONFINITE);
}

// One sub-batch, persistent grid over the resident CTAs in clusters of
// C = crun.  Phase 1 (C > 1): each cluster takes the next of the first
// nbig cells of `order` (the largest) and solves it with all its CTAs
// (cell_solve_dist).  Phase 2: every CTA takes the remaining cells one at a
// time (cell_solve_body on one CTA).  The order (largest estimated work first
// within each phase, k_cell_order) only decides when a cell starts; the
// results do not depend on it.
// `crun`: the cluster size of the sub-batch's main grid (<= S.dist_c; k_cell_order
// classified the cells for it); `cluster`: this launch's -- crun for the main
// grid, 1 for a helper grid that runs phase 2 only on the SMs the clusters
// leave idle (both take phase-2 cells from the same queue).
template <typename R>
__global__ void __launch_bounds__(kCellThreads, 1)
k_cell_solve(DevState S, const CellDesc* __restrict__ cells, const int* __restrict__ order,
             const int* __restrict__ nbig_p, int begin, int nbatch, int crun, int cluster) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int sj;
  if (*(volatile int*)S.status & ST_HALT) {   // halted until the host reruns the sub-batch
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nbatch; j += gridDim.x * blockDim.x)
      S.cout[j].status = CELL_SKIPPED;
    return;
  }
  const int C = cluster;
  const int nbig = (crun > 1 && order) ? *nbig_p : 0;
  if (C > 1) {
    const int crank = (int)cg::this_cluster().block_rank();
    // every CTA of the cluster must have started before one writes another's shared memory
    cg::this_cluster().sync();
    for (;;) {
      if (crank == 0 && threadIdx.x == 0) {
        const int j = (int)atomicAdd(S.queue, 1u);
        for (int r = 0; r < C; ++r) *cg::this_cluster().map_shared_rank(&sj, r) = j;
      }
      cg::this_cluster().sync();
      const int j = sj;
      if (j >= nbig) break;
      const int cidx = order[begin + j];
      cell_solve_dist<R>(S, cells[begin + cidx], cidx, nbatch, crank, C, smem_raw);
      cg::this_cluster().sync();
    }
  }
  // no shared memory of another CTA is touched from here on
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sj = (int)atomicAdd(S.queue + 1, 1u);
    __syncthreads();
    const int j = nbig + sj;
    if (j >= nbatch) break;
    const int cidx = order ? order[begin + j] : j;
    cell_solve_body<R>(S, cells[begin + cidx], cidx, nbatch, smem_raw);
  }
}

// Estimated work of one cell solve iteration: the exp terms of the four
// separable passes, nx1 nx2 (W + H) + H W (nx1 + nx2), from the member boxes;
// H, W: the cell's Y box.
__device__ __forceinline__ unsigned int cell_cost(const DevState& S, const CellDesc& cd, int* Hout, int* Wout) {
  int k0 = 1 << 30, l0 = 1 << 30, k1 = -1, l1 = -1;
  for (int q = 0; q < 4; ++q) {
    if (cd.mem[q] < 0) continue;
    const BoxRec b = S.box[cd.mem[q]];
    if (b.H * b.W == 0) continue;
    k0 = min(k0, b.k0); l0 = min(l0, b.l0);
    k1 = max(k1, b.k0 + b.H); l1 = max(l1, b.l0 + b.W);
  }
  if (k1 < 0) {
    *Hout = *Wout = 0;
    return 1u;
  }
  const long long H = min(S.N, k1 + S.margin) - max(0, k0 - S.margin);
  const long long W = min(S.N, l1 + S.margin) - max(0, l0 - S.margin);
  *Hout = (int)H;
  *Wout = (int)W;
  const long long c = (long long)cd.nx1 * cd.nx2 * (W + H) + H * W * (cd.nx1 + cd.nx2);
  return (unsigned int)min(c + 1, 0x7fffffffLL);
}

// Whether a cell with Y box H x W fits a cluster of the layout's largest size
// (S.dist_c CTAs, each holding a block of ceil(H / dist_c) rows).
__device__ __forceinline__ bool fits_layout(const DevState& S, int H, int W) {
  if (S.dist_c < 2) return false;
  const int hl = (H + S.dist_c - 1) / S.dist_c;
  return H >= S.dist_c && W <= S.dist_cap_w && hl <= S.dist_cap_hl && hl * W <= S.dist_cap_nyl;
}

constexpr int kOrderMax = 4096;   // largest batch sorted (larger ones keep their index order)

// Order of the cells of each sub-batch of partition `part` (block b:
// sub-batch b; one block for the whole partition when not staggered) and the
// number of leading cells that a whole cluster of C CTAs solves.  mode 0: a
// cell goes to a cluster if it fits the cluster layout and either does not fit
// one CTA or its work exceeds `factor` times the mean work per CTA (`slots`
// CTAs); mode 1:
// every cell that fits the cluster layout; mode 2: none.  Within each group
// the cells are sorted by decreasing work (bitonic sort of (group, cost,
// index) keys in shared memory; ties keep the index order).
__global__ void __launch_bounds__(1024) k_cell_order(DevState S, int part, int mode, int slots, int C,
                                                     double factor) {
  __shared__ unsigned long long key[kOrderMax];
  __shared__ double red[33];
  const int b = blockIdx.x;
  const int begin = S.staggered ? S.sub_start[part][b] : 0;
  const int end = S.staggered ? S.sub_start[part][b + 1] : S.sub_start[part][4];
  const int n = end - begin;
  int* out = S.order[part] + begin;
  int* nbig = S.nbig + part * 4 + b;
  if (*(volatile int*)S.status & ST_HALT) return;   // the sweep's cell launches solve nothing
  if (n <= 0) {
    if (threadIdx.x == 0) *nbig = 0;
    return;
  }
  int P = 1;
  while (P < n) P <<= 1;
  if (P > kOrderMax) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = i;
    if (threadIdx.x == 0) *nbig = 0;
    return;
  }
  const CellDesc* cells = S.cells[part];
  double tot[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    int H, W;
    tot[0] += (double)cell_cost(S, cells[begin + i], &H, &W);
  }
  block_sum<1>(tot, red);
  const double thr = factor * tot[0] / (double)max(1, slots);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long k = 0ull;
    if (i < n) {
      int H, W;
      const unsigned int cost = cell_cost(S, cells[begin + i], &H, &W);
      const int hl = C > 0 ? (H + C - 1) / C : H;
      const bool fits_dist = C > 1 && C <= S.dist_c && H >= C && W <= S.dist_cap_w && hl <= S.dist_cap_hl &&
                             hl * W <= S.dist_cap_nyl;
      const bool fits_one = H <= S.cap_side && W <= S.cap_side && H * W <= S.cap_ny;
      const bool big = mode != 2 && fits_dist && (mode == 1 || !fits_one || (double)cost > thr);
      if (!fits_one && !big && fits_layout(S, H, W) && (mode == 2 || C < S.dist_c)) atomicOr(S.status, ST_REGROUP);
      k = ((unsigned long long)big << 62) | ((unsigned long long)cost << 30) | (0x3fffffffu - (unsigned)i);
    }
    key[i] = k;
  }
  __syncthreads();
  // descending bitonic sort
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], c = key[ixj];
          const bool first_half = (i & k) == 0;
          if (first_half ? (a < c) : (a > c)) { key[i] = c; key[ixj] = a; }
        }
      }
      __syncthreads();
    }
  int cnt = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    out[i] = (int)(0x3fffffffu - (unsigned)(key[i] & 0x3fffffffull));
    cnt += (int)((key[i] >> 62) & 1ull);
  }
  double cv[1] = {(double)cnt};
  block_sum<1>(cv, red);
  if (threadIdx.x == 0) *nbig = (int)cv[0];
}

cudaError_t launch_cell_order(const DevState& S, int part, int mode, int slots, int C, double factor,
                              cudaStream_t st) {
  k_cell_order<<<S.staggered ? 4 : 1, 1024, 0, st>>>(S, part, mode, slots, C, factor);
  return cudaGetLastError();
}

// Many independent instances, one staggered sub-batch of every instance per
// launch: the same two phases as k_cell_solve over the (instance, cell)
// references in the order of k_ref_order -- clusters of C CTAs take the first
// nbig references (each CTA loads that instance's state), then every CTA takes
// the rest one at a time.  C must not exceed any instance's dist_c (its
// cluster layout was sized for dist_c CTAs).
template <typename R>
__global__ void __launch_bounds__(kCellThreads, 1)
k_cell_solve_multi(const DevState* __restrict__ states, const CellRef* __restrict__ refs,
                   const int* __restrict__ order, const int* __restrict__ nbig_p, int nref, int part,
                   unsigned int* queue, int C) {
  namespace cg = cooperative_groups;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ DevState sS;
  __shared__ int sj;
  auto load_state = [&](int inst) {
    const int* src = reinterpret_cast<const int*>(states + inst);
    int* dst = reinterpret_cast<int*>(&sS);
    for (int w = threadIdx.x; w < (int)(sizeof(DevState) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
  };
  // a halted instance (status read once per reference, the same in every CTA
  // of a cluster) solves nothing: its cell is marked skipped
  auto halted = [&](const CellRef& rf) {
    if (!(*(volatile int*)sS.status & ST_HALT)) return false;
    if (threadIdx.x == 0 && (C == 1 || (int)cg::this_cluster().block_rank() == 0))
      sS.cout[rf.pos].status = CELL_SKIPPED;
    return true;
  };
  const int nbig = C > 1 ? *nbig_p : 0;
  if (C > 1) {
    const int crank = (int)cg::this_cluster().block_rank();
    // every CTA of the cluster must have started before one writes another's shared memory
    cg::this_cluster().sync();
    for (;;) {
      if (crank == 0 && threadIdx.x == 0) {
        const int j = (int)atomicAdd(queue, 1u);
        for (int r = 0; r < C; ++r) *cg::this_cluster().map_shared_rank(&sj, r) = j;
      }
      cg::this_cluster().sync();
      const int j = sj;
      if (j >= nbig) break;
      const CellRef rf = refs[order[j]];
      load_state(rf.inst);
      if (!halted(rf)) cell_solve_dist<R>(sS, sS.cells[part][rf.cell], rf.pos, rf.nbatch, crank, C, smem_raw);
      cg::this_cluster().sync();
    }
  }
  // no shared memory of another CTA is touched from here on
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sj = (int)atomicAdd(queue + 1, 1u);
    __syncthreads();
    const int j = nbig + sj;
    if (j >= nref) break;
    const CellRef rf = refs[order ? order[j] : j];
    load_state(rf.inst);
    if (!halted(rf)) cell_solve_body<R>(sS, sS.cells[part][rf.cell], rf.pos, rf.nbatch, smem_raw);
  }
}

constexpr int kRefOrderMax = 8192;   // largest reference list sorted (longer ones keep their order)

// Order of the nref references of one many-instance launch (one block): cluster
// references first -- those whose box fits the instance's cluster layout for C
// CTAs and whose estimated work exceeds `factor` times the mean work per CTA
// (`slots` CTAs), or that do not fit one CTA -- each group by decreasing
// estimated work (as k_cell_order); *nbig = the number of cluster references.
__global__ void __launch_bounds__(1024)
k_ref_order(const DevState* __restrict__ states, const CellRef* __restrict__ refs, int nref, int part, int C,
            double factor, int slots, int* order, int* nbig) {
  extern __shared__ unsigned long long rkey[];
  __shared__ double red[33];
  int P = 1;
  while (P < nref) P <<= 1;
  if (P > kRefOrderMax) {
    for (int i = threadIdx.x; i < nref; i += blockDim.x) order[i] = i;
    if (threadIdx.x == 0) *nbig = 0;
    return;
  }
  double tot[1] = {0.0};
  for (int i = threadIdx.x; i < nref; i += blockDim.x) {
    const CellRef rf = refs[i];
    int H, W;
    tot[0] += (double)cell_cost(states[rf.inst], states[rf.inst].cells[part][rf.cell], &H, &W);
  }
  block_sum<1>(tot, red);
  const double thr = factor * tot[0] / (double)max(1, slots);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long k = 0ull;
    if (i < nref) {
      const CellRef rf = refs[i];
      const DevState& S = states[rf.inst];
      int H, W;
      const unsigned int cost = cell_cost(S, S.cells[part][rf.cell], &H, &W);
      const int hl = (H + C - 1) / C;
      const bool fits_dist = C > 1 && C <= S.dist_c && H >= C && W <= S.dist_cap_w && hl <= S.dist_cap_hl &&
                             hl * W <= S.dist_cap_nyl;
      const bool fits_one = H <= S.cap_side && W <= S.cap_side && H * W <= S.cap_ny;
      const bool big = fits_dist && (!fits_one || (double)cost > thr);
      if (!fits_one && !big && fits_layout(S, H, W) && C < S.dist_c) atomicOr(S.status, ST_REGROUP);
      k = ((unsigned long long)big << 62) | ((unsigned long long)cost << 30) | (0x3fffffffu - (unsigned)i);
    }
    rkey[i] = k;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = rkey[i], c = rkey[ixj];
          const bool first_half = (i & k) == 0;
          if (first_half ? (a < c) : (a > c)) { rkey[i] = c; rkey[ixj] = a; }
        }
      }
      __syncthreads();
    }
  int cnt = 0;
  for (int i = threadIdx.x; i < nref; i += blockDim.x) {
    order[i] = (int)(0x3fffffffu - (unsigned)(rkey[i] & 0x3fffffffull));
    cnt += (int)((rkey[i] >> 62) & 1ull);
  }
  double cv[1] = {(double)cnt};
  block_sum<1>(cv, red);
  if (threadIdx.x == 0) *nbig = (int)cv[0];
}

size_t cell_smem_bytes(int s, int cap_side, int cap_ny, int precision) {
  size_t rs = precision ? sizeof(double) : sizeof(float);
  size_t cap_nx = 4 * (size_t)s * s, tsz = 2 * (size_t)s * cap_side;
  return 32 * 16 * sizeof(double) + rs * (7 * cap_nx + 2 * tsz + 5 * (size_t)cap_ny);
}

// Shared memory of the cluster-distributed layout (cell_solve_dist).
size_t dist_smem_bytes(int s, int C, int cap_w, int cap_hl, int cap_nyl, int precision) {
  const size_t rs = precision ? sizeof(double) : sizeof(float), cap_nx = 4 * (size_t)s * s;
  return 32 * 16 * sizeof(double) +
         rs * ((8 + (size_t)C) * cap_nx + 2 * (size_t)s * cap_w + 2 * (size_t)s * cap_hl + 5 * (size_t)cap_nyl);
}

// Static shared memory of the cell kernels, the larger of the single- and the
// many-instance kernel (the dynamic part must leave room for it).
int cell_static_smem(int precision) {
  cudaFuncAttributes a1, a2;
  cudaError_t e1 = precision ? cudaFuncGetAttributes(&a1, k_cell_solve<double>)
                             : cudaFuncGetAttributes(&a1, k_cell_solve<float>);
  cudaError_t e2 = precision ? cudaFuncGetAttributes(&a2, k_cell_solve_multi<double>)
                             : cudaFuncGetAttributes(&a2, k_cell_solve_multi<float>);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return 4096;
  }
  return (int)std::max(a1.sharedSizeBytes, a2.sharedSizeBytes);
}

// Resident CTAs of the single-instance cell kernel with `smem` dynamic bytes:
// C == 1 single CTAs, C > 1 the CTAs of the resident C-CTA clusters (0 if such
// clusters cannot be scheduled).
int cell_resident_ctas(size_t smem, int C, int precision) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (precision) e = cudaFuncSetAttribute(k_cell_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else e = cudaFuncSetAttribute(k_cell_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C <= 1) {
    int per = 0;
    e = precision ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell_solve<double>, kCellThreads, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell_solve<float>, kCellThreads, smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nsm > 0 ? nsm : 1;
    }
    return std::max(1, per * nsm);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCellThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = precision ? cudaOccupancyMaxActiveClusters(&n, k_cell_solve<double>, &cfg)
                : cudaOccupancyMaxActiveClusters(&n, k_cell_solve<float>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n * C;
}

// One sub-batch: `nctas` persistent CTAs (a multiple of `cluster`, at most the
// resident ones) in clusters of `cluster` (the main grid: crun), `smem` dynamic
// bytes; cluster = 1 with crun > 1 launches single CTAs that run phase 2 only.
cudaError_t launch_cell_solve(const DevState& S, const CellDesc* cells, const int* order, const int* nbig_p,
                              int begin, int nbatch, int precision, size_t smem, int nctas, int crun, int cluster,
                              cudaStream_t st) {
  const int C = std::max(1, cluster);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(C, nctas / C * C));
  cfg.blockDim = dim3(kCellThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = C > 1 ? 1 : 0;
  if (precision) {
    cudaFuncSetAttribute(k_cell_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaLaunchKernelEx(&cfg, k_cell_solve<double>, S, cells, order, nbig_p, begin, nbatch, crun, C);
  }
  cudaFuncSetAttribute(k_cell_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaLaunchKernelEx(&cfg, k_cell_solve<float>, S, cells, order, nbig_p, begin, nbatch, crun, C);
}

// One many-instance launch: order the references (k_ref_order), then `nctas`
// persistent CTAs (a multiple of C) in clusters of C; `order` and `nbig` are
// device scratch (nref ints, one int), `queue` two counters.
cudaError_t launch_cell_solve_multi(const DevState* states, const CellRef* refs, int nref, int part, int* order,
                                    int* nbig, unsigned int* queue, size_t smem, int precision, int C,
                                    double factor, int nctas, cudaStream_t st) {
  C = std::max(1, C);
  int P = 1;
  while (P < nref) P <<= 1;
  const size_t osm = (size_t)std::min(P, kRefOrderMax) * sizeof(unsigned long long);
  cudaFuncSetAttribute(k_ref_order, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)osm);
  k_ref_order<<<1, 1024, osm, st>>>(states, refs, nref, part, C, factor, nctas, order, nbig);
  cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned int), st);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(C, nctas / C * C));
  cfg.blockDim = dim3(kCellThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = C > 1 ? 1 : 0;
  if (precision) {
    cudaFuncSetAttribute(k_cell_solve_multi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaLaunchKernelEx(&cfg, k_cell_solve_multi<double>, states, refs, (const int*)order, (const int*)nbig,
                              nref, part, queue, C);
  }
  cudaFuncSetAttribute(k_cell_solve_multi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaLaunchKernelEx(&cfg, k_cell_solve_multi<float>, states, refs, (const int*)order, (const int*)nbig, nref,
                            part, queue, C);
}

// Resident CTAs of the many-instance kernel in clusters of C (0: not schedulable).
int cell_multi_resident_ctas(size_t smem, int C, int precision) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = precision
                      ? cudaFuncSetAttribute(k_cell_solve_multi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem)
                      : cudaFuncSetAttribute(k_cell_solve_multi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (C <= 1) {
    int per = 0;
    e = precision ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell_solve_multi<double>, kCellThreads, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cell_solve_multi<float>, kCellThreads, smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return nsm;
    }
    return std::max(1, per * nsm);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCellThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = precision ? cudaOccupancyMaxActiveClusters(&n, k_cell_solve_multi<double>, &cfg)
                : cudaOccupancyMaxActiveClusters(&n, k_cell_solve_multi<float>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n * C;
}
