// Global unbalanced Sinkhorn on the N x N grid (Eq. sinkhorn-iters-ot, nu_- = 0):
// the comparator of Section 5.3, the warm start of DomDec, and the global
// log-sum-exp of the primal-dual certificate.
//
// A half-step needs, for every x, L(x) = log sum_y exp(f(y) - |x-y|^2/eps) with
// f = pot/eps + log m.  Two evaluations:
//  * dense      : all N^2 terms per x (the plain method), f tiled through shared memory;
//  * separable  : |x-y|^2 = (x1-y1)^2 + (x2-y2)^2, so L is a 1-D log-sum-exp along rows
//                 followed by one along columns: 2 N^3 terms instead of N^4.
// Values are kept in log2 units (ex2/lg2); float or double arithmetic.
#include <cmath>

#include "dd_common.cuh"
#include "domdec.h"

namespace {

// Terms more than `cut` (log2 units) below the maximum are skipped: at most N
// of them change the sum by N 2^-cut relative (< 1e-15 in double, < 1e-7 in float).
template <typename R> __device__ __forceinline__ R cut_log2() { return sizeof(R) == 4 ? R(32) : R(64); }

// One 1-D log-sum-exp per target with P lanes: the maximum and the window
// test run in float on the shadow values; only terms within `cut` of the
// maximum are evaluated (in R) and summed.
// FAST (double only): each kept term's exponent is formed in double and only its
// exponential (at most `cut` below the maximum) is taken in float (ex2.approx);
// the sums stay double.  The sum's relative error is ~1e-7, i.e. ~1e-7 absolute
// in log2 units, whatever the magnitude of the exponents.
template <typename R, bool FAST = false, typename FS, typename FF>
__device__ __forceinline__ R lse_window(FS src, FF srcf, int M, int ctr, double q2, int part, int P) {
  const float q2f = (float)q2;
  float mxf = -INFINITY;
  for (int m = part; m < M; m += P) {
    float d = (float)(ctr - m);
    mxf = fmaxf(mxf, srcf(m) - q2f * d * d);
  }
  for (int o = 1; o < P; o <<= 1) mxf = fmaxf(mxf, __shfl_xor_sync(0xffffffffu, mxf, o));
  if (!(mxf > -INFINITY)) return R(mxf);
  const float cutf = (float)cut_log2<R>() + 1.0f;
  const R mx = R(mxf), q2r = R(q2);
  R acc = R(0);
  for (int m = part; m < M; m += P) {
    float d = (float)(ctr - m);
    if (srcf(m) - q2f * d * d - mxf > -cutf) {
      R dr = R(ctr - m);
      if (FAST) acc += R(dd_ex2(float(src(m) - q2r * dr * dr - mx)));
      else acc += dd_ex2(src(m) - q2r * dr * dr - mx);
    }
  }
  for (int o = 1; o < P; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return mx + dd_lg2(acc);
}

// The same log-sum-exp against a shift `sig` (the previous iteration's value of
// this target) in one pass: terms more than `cut` below the shift are skipped,
// so the skipped mass is below N 2^-cut of the sum, as for the max-shifted
// window.  When the shift is unusable -- NaN, a term more than 60 above it,
// or a sum outside [2^-30, 2^60] -- the lane group falls back to lse_window
// (warp-collective: every lane of the warp runs the fallback if one group needs it).
template <typename R, bool FAST = false, typename FS, typename FF>
__device__ __forceinline__ R lse_window_shift(FS src, FF srcf, int M, int ctr, double q2, int part, int P, R sig) {
  const float q2f = (float)q2, sigf = (float)sig;
  const float cutf = (float)cut_log2<R>() + 1.0f;
  const R q2r = R(q2);
  R acc = R(0);
  bool bad = !(sigf > -INFINITY && sigf < INFINITY);
  if (!bad) {
    for (int m = part; m < M; m += P) {
      const float d = (float)(ctr - m);
      const float vf = srcf(m) - q2f * d * d - sigf;
      if (vf > -cutf) {
        bad |= vf > 60.0f;
        const R dr = R(ctr - m);
        if (FAST) acc += R(dd_ex2(float(src(m) - q2r * dr * dr - sig)));
        else acc += dd_ex2(src(m) - q2r * dr * dr - sig);
      }
    }
  }
  for (int o = 1; o < P; o <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    bad |= __shfl_xor_sync(0xffffffffu, (int)bad, o) != 0;
  }
  bad |= !(acc >= R(9.313225746154785e-10) && acc <= R(1.152921504606847e18));   // [2^-30, 2^60]
  if (__any_sync(0xffffffffu, bad)) {
    const R v = lse_window<R, FAST>(src, srcf, M, ctr, q2, part, P);
    if (bad) return v;
  }
  return sig + dd_lg2(acc);
}

constexpr int kSepLanes = 4;   // lanes per target in the separable passes

// Row pass with a transposed store: dst[j*N + k] = log2 sum_l 2^{src[k*N + l] - q2 (j - l)^2}
// (block = row k).  Applied twice it gives the 2-D log-sum-exp in the original
// layout (the second pass runs along the columns of the original image), with
// every source read from shared memory instead of strided global loads.
// With `shifted`, dst holds the previous iteration's values on entry and each
// target is evaluated in one pass against its previous value
// (lse_window_shift); otherwise max-shifted (lse_window).
template <typename R, bool FAST>
__global__ void __launch_bounds__(1024)
k_sep_rows_t(const R* __restrict__ src, const float* __restrict__ srcf, R* dst,
             float* __restrict__ dstf, int N, double q2, int shifted) {
  extern __shared__ __align__(16) unsigned char sm[];
  R* row = reinterpret_cast<R*>(sm);
  float* rowf = reinterpret_cast<float*>(row + N);
  const int k = blockIdx.x;
  for (int l = threadIdx.x; l < N; l += blockDim.x) {
    row[l] = src[(long long)k * N + l];
    rowf[l] = srcf[(long long)k * N + l];
  }
  __syncthreads();
  const int P = kSepLanes, nt = (N * P + 31) & ~31;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    const int j0 = i / P, part = i % P, j = min(j0, N - 1);
    auto srcv = [&](int m) { return row[m]; };
    auto srcfv = [&](int m) { return rowf[m]; };
    R v;
    if (shifted) v = lse_window_shift<R, FAST>(srcv, srcfv, N, j, q2, part, P, dst[(long long)j * N + k]);
    else v = lse_window<R, FAST>(srcv, srcfv, N, j, q2, part, P);
    __syncwarp();
    if (part == 0 && j0 < N) {
      dst[(long long)j * N + k] = v;
      if (dstf) dstf[(long long)j * N + k] = (float)v;
    }
  }
}

// Dense: out[x] = log2 sum_y 2^{in[y] - q2 |x - y|^2}, shifted by the previous
// value out[x] when `use_shift` (one pass), exact max-shifted otherwise.
template <typename R>
__global__ void __launch_bounds__(256) k_dense(const R* __restrict__ in, R* __restrict__ out, int N, R q2,
                                               int use_shift) {
  constexpr int TILE = 1024;
  __shared__ R tile[TILE];
  const int n = N * N;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const R x1 = R(x / N), x2 = R(x % N);
  const bool active = x < n;
  R shift = (active && use_shift) ? out[x] : R(0);
  bool exact = !use_shift;
  R acc = R(0), mx = -dd_inf<R>();
  for (int pass = 0; pass < 3; ++pass) {
    // pass 0: shifted sum (if use_shift); pass 1: max (if exact); pass 2: sum (if exact)
    if (pass == 0 && !use_shift) continue;
    if (pass > 0) {
      int need = __syncthreads_or(active && exact);
      if (!need) break;
    }
    for (int t0 = 0; t0 < n; t0 += TILE) {
      __syncthreads();
      for (int t = threadIdx.x; t < TILE && t0 + t < n; t += blockDim.x) tile[t] = in[t0 + t];
      __syncthreads();
      if (!active || (pass > 0 && !exact)) continue;
      const int cnt = min(TILE, n - t0);
      for (int t = 0; t < cnt; ++t) {
        int y = t0 + t;
        R d1 = x1 - R(y / N), d2 = x2 - R(y % N);
        R v = tile[t] - q2 * (d1 * d1 + d2 * d2);
        if (pass == 0) acc += dd_ex2(v - shift);
        else if (pass == 1) mx = max(mx, v);
        else acc += dd_ex2(v - mx);
      }
    }
    if (pass == 0 && active) {
      if (acc > R(1e-25) && acc < R(1e25)) shift = shift + dd_lg2(acc);
      else { exact = true; acc = R(0); }
    }
  }
  if (active) out[x] = exact ? (mx > -dd_inf<R>() ? mx + dd_lg2(acc) : mx) : shift;
}

template <typename R>
__global__ void k_to_log2(const double* __restrict__ pot, const double* __restrict__ logm, double inv_eps,
                          R* __restrict__ out, int n, float* __restrict__ shadow = nullptr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    R v = R((pot ? pot[i] * inv_eps : 0.0) + logm[i]) * R(DD_LOG2E);
    out[i] = v;
    if (shadow) shadow[i] = (float)v;
  }
}

template <typename R>
__global__ void k_half(const R* __restrict__ lse2, double kappa, double* __restrict__ pot, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pot[i] = -kappa * (double)lse2[i] * DD_LN2;
}

template <typename R>
__global__ void k_to_nat(const R* __restrict__ lse2, double* __restrict__ out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (double)lse2[i] * DD_LN2;
}

// PD/lam = KL(P_X | e^{-alpha/lam} mu) with P_X = mu e^{alpha/eps + w} (Eq. PD-gap-KL).
// And the dual of Eq. dual-problem: out = [gap, sum_y nu e^{beta/eps + z}, conj terms..., |mu|, |nu|]
template <typename R>
__global__ void __launch_bounds__(512)
k_sk_eval(const double* __restrict__ mu, const double* __restrict__ nu, const double* __restrict__ alpha,
          const double* __restrict__ beta, const R* __restrict__ w2, const R* __restrict__ z2, double eps,
          double lam, int n, double* out) {
  __shared__ double red[33 * 6];
  double v[6] = {0, 0, 0, 0, 0, 0};
  const bool fin = isfinite(lam);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double a = alpha[i], m = mu[i];
    double t = a / eps + (double)w2[i] * DD_LN2;  // log(P_X/mu)
    double g = fin ? -a / lam : 0.0;              // log(e^{-alpha/lam})
    v[0] += m * exp(g) * dd_psi<double>(t - g);
    if (z2) {
      double b = beta[i], z = (double)z2[i] * DD_LN2;
      v[1] += nu[i] * exp(b / eps + z);
      v[2] += fin ? lam * (exp(-a / lam) - 1.0) * m : -a * m;
      v[3] += fin ? lam * (exp(-b / lam) - 1.0) * nu[i] : -b * nu[i];
    }
    v[4] += m;
    v[5] += nu[i];
  }
  block_sum_to<6>(v, red, out);
}

// k_sk_eval over the grid; partials: kRedBlocks * 6 doubles (NULL: one block).
template <typename R>
void sk_eval(const double* mu, const double* nu, const double* alpha, const double* beta, const R* w2,
             const R* z2, double eps, double lam, int n, double* d_eval, double* partials, cudaStream_t st) {
  const int G = red_blocks(n, 512, partials);
  if (G == 1) {
    k_sk_eval<R><<<1, 512, 0, st>>>(mu, nu, alpha, beta, w2, z2, eps, lam, n, d_eval);
  } else {
    k_sk_eval<R><<<G, 512, 0, st>>>(mu, nu, alpha, beta, w2, z2, eps, lam, n, partials);
    k_sum_partials<<<1, 32, 0, st>>>(partials, G, 6, d_eval);
  }
}

// Translation step (optional, not in the paper): after an X-half,
// alpha += (lam/2) log(<e^{-alpha/lam}, mu> / <e^{-beta/lam}, nu>), the maximiser
// of the dual of Eq. dual-problem along (alpha + t, beta - t).
__global__ void __launch_bounds__(512) k_ti_sums(const double* __restrict__ mu, const double* __restrict__ nu,
                                                 const double* __restrict__ alpha, const double* __restrict__ beta,
                                                 double lam, int n, double* out) {
  __shared__ double red[33 * 2];
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[0] += mu[i] * exp(-alpha[i] / lam);
    v[1] += nu[i] * exp(-beta[i] / lam);
  }
  block_sum_to<2>(v, red, out);
}

__global__ void k_ti_apply(double* __restrict__ alpha, const double* __restrict__ sums, double lam, int n) {
  const double t = 0.5 * lam * log(sums[0] / sums[1]);
  if (!(t == t) || isinf(t)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) alpha[i] += t;
}

// sums: 2 doubles of device scratch; partials: kRedBlocks * 2 doubles.
void ti_step(const double* mu, const double* nu, double* alpha, const double* beta, double lam, int n,
             double* sums, double* partials, cudaStream_t st) {
  const int G = red_blocks(n, 512, partials);
  k_ti_sums<<<G, 512, 0, st>>>(mu, nu, alpha, beta, lam, n, partials);
  k_sum_partials<<<1, 32, 0, st>>>(partials, G, 2, sums);
  k_ti_apply<<<(n + 255) / 256, 256, 0, st>>>(alpha, sums, lam, n);
}

template <typename R>
struct Work {
  R *in2, *tmp, *w2, *z2, *tmpz;
  float *in2f, *tmpf;  // float shadows (double precision only)
};

// in2f / tmpf: float shadows (required for R = double; ignored for float).
// use_shift (separable): tmp and out2 hold this evaluation's previous values
// (tmp: the row pass, transposed) and every target is summed against them in
// one pass; otherwise max-shifted.
template <typename R>
cudaError_t lse_all(const R* in2, R* tmp, R* out2, int N, double q, int variant, int use_shift, cudaStream_t st,
                    const float* in2f = nullptr, float* tmpf = nullptr, bool fast = false) {
  if (variant == 1) {
    const float* inf = sizeof(R) == 8 ? in2f : reinterpret_cast<const float*>(in2);
    float* tf = sizeof(R) == 8 ? tmpf : nullptr;                       // shadow written by pass 1
    const float* tfr = sizeof(R) == 8 ? tmpf : reinterpret_cast<const float*>(tmp);
    const double q2 = q * DD_LOG2E;
    const int thr_rows = min(1024, ((N * kSepLanes + 31) / 32) * 32);
    const size_t sm = N * (sizeof(R) + sizeof(float));
    // rows, stored transposed; then the rows of that (the original columns), transposed back
    const int sh = use_shift ? 1 : 0;
    if (fast && sizeof(R) == 8) {
      k_sep_rows_t<R, true><<<N, thr_rows, sm, st>>>(in2, inf, tmp, tf, N, q2, sh);
      k_sep_rows_t<R, true><<<N, thr_rows, sm, st>>>(tmp, tfr, out2, nullptr, N, q2, sh);
    } else {
      k_sep_rows_t<R, false><<<N, thr_rows, sm, st>>>(in2, inf, tmp, tf, N, q2, sh);
      k_sep_rows_t<R, false><<<N, thr_rows, sm, st>>>(tmp, tfr, out2, nullptr, N, q2, sh);
    }
  } else {
    R q2 = R(q * DD_LOG2E);
    int n = N * N;
    k_dense<R><<<(n + 255) / 256, 256, 0, st>>>(in2, out2, N, q2, use_shift);
  }
  return cudaGetLastError();
}

}  // namespace

// Separable FP64 log-sum-exp over the whole grid (natural units):
// out[x] = log sum_y exp(pot[y]/eps + logm[y] - h^2 |x-y|^2/eps).  pot may be NULL.
// buf_a, buf_b, buf_c: N*N doubles of scratch each.
cudaError_t global_lse64(const double* pot, const double* logm, double eps, double h, int N, double* out,
                         double* buf_a, double* buf_b, double* buf_c, cudaStream_t st) {
  int n = N * N;
  float* sh_in = reinterpret_cast<float*>(buf_c);
  float* sh_tmp = sh_in + n;
  k_to_log2<double><<<(n + 255) / 256, 256, 0, st>>>(pot, logm, 1.0 / eps, buf_a, n, sh_in);
  lse_all<double>(buf_a, buf_b, buf_a, N, h * h / eps, 1, 0, st, sh_in, sh_tmp);
  k_to_nat<double><<<(n + 255) / 256, 256, 0, st>>>(buf_a, out, n);
  return cudaGetLastError();
}

// Full Sinkhorn driver; all pointers device.  Returns 0, or 1 when the last
// stage hit maxit.  out: [iterations, PD/lam, primal, dual].
template <typename R>
static int full_sinkhorn_impl(const double* mu, const double* nu, const double* logmu, const double* lognu,
                              int N, double eps_start, double eps, double lam, int variant, int maxit,
                              double err, int check_every, double* alpha, double* beta, double* out,
                              double* d_eval, cudaStream_t st, cudaError_t* cerr, bool fast = false) {
  const int n = N * N;
  const double h = 1.0 / N;
  const bool ti = (variant & DOMDEC_SINKHORN_TI) && std::isfinite(lam);
  variant &= ~DOMDEC_SINKHORN_TI;
  Work<R> w;
  const size_t wbytes = (sizeof(R) * 5 * (size_t)n + sizeof(float) * 2 * (size_t)n + 255) & ~size_t(255);
  *cerr = cudaMallocAsync(&w.in2, wbytes + sizeof(double) * 6 * kRedBlocks, st);
  if (*cerr != cudaSuccess) return -1;
  // row-pass results of the two half-steps kept apart (each is the next shift of its own half-step)
  w.tmp = w.in2 + n; w.w2 = w.tmp + n; w.z2 = w.w2 + n; w.tmpz = w.z2 + n;
  w.in2f = reinterpret_cast<float*>(w.tmpz + n);
  w.tmpf = w.in2f + n;
  double* partials = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(w.in2) + wbytes);
  const int grid = (n + 255) / 256;
  double evalh[6];
  long long total = 0;
  double gap = INFINITY;
  int rc = 0;
  if (check_every < 1) check_every = 1;
  double e = eps_start > eps ? eps_start : eps;
  bool first_stage = true;
  for (;;) {
    const double kap = std::isfinite(lam) ? e / (1.0 + e / lam) : e;
    const double q = h * h / e;
    // w = LSE_y[beta/e + log nu]
    k_to_log2<R><<<grid, 256, 0, st>>>(beta, lognu, 1.0 / e, w.in2, n, w.in2f);
    lse_all<R>(w.in2, w.tmp, w.w2, N, q, variant, 0, st, w.in2f, w.tmpf, fast);
    int it = 0;
    bool conv = false;
    int shift_ok = 0;
    while (it < maxit) {
      k_half<R><<<grid, 256, 0, st>>>(w.w2, kap, alpha, n);
      if (ti) ti_step(mu, nu, alpha, beta, lam, n, d_eval + 6, partials, st);
      k_to_log2<R><<<grid, 256, 0, st>>>(alpha, logmu, 1.0 / e, w.in2, n, w.in2f);
      lse_all<R>(w.in2, w.tmpz, w.z2, N, q, variant, shift_ok, st, w.in2f, w.tmpf, fast);
      k_half<R><<<grid, 256, 0, st>>>(w.z2, kap, beta, n);
      k_to_log2<R><<<grid, 256, 0, st>>>(beta, lognu, 1.0 / e, w.in2, n, w.in2f);
      lse_all<R>(w.in2, w.tmp, w.w2, N, q, variant, 1, st, w.in2f, w.tmpf, fast);
      shift_ok = 1;
      ++it;
      if (it % check_every == 0 || it == maxit) {
        sk_eval<R>(mu, nu, alpha, beta, w.w2, nullptr, e, lam, n, d_eval, partials, st);
        cudaMemcpyAsync(evalh, d_eval, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
        *cerr = cudaStreamSynchronize(st);
        if (*cerr != cudaSuccess) { cudaFreeAsync(w.in2, st); return -1; }
        gap = evalh[0];
        if (err >= 0.0 && gap <= err * evalh[4]) { conv = true; break; }
        if (!(gap == gap)) break;
      }
    }
    total += it;
    first_stage = false;
    (void)first_stage;
    if (e <= eps) { rc = conv || err < 0.0 ? 0 : 1; break; }
    e = fmax(eps, 0.5 * e);
  }
  // primal / dual at the final eps (z from the last Y-half of the final iterate)
  const double kap = std::isfinite(lam) ? eps / (1.0 + eps / lam) : eps;
  (void)kap;
  sk_eval<R>(mu, nu, alpha, beta, w.w2, w.z2, eps, lam, n, d_eval, partials, st);
  cudaMemcpyAsync(evalh, d_eval, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  *cerr = cudaStreamSynchronize(st);
  cudaFreeAsync(w.in2, st);
  if (*cerr != cudaSuccess) return -1;
  const double D = eps * evalh[4] * evalh[5] - eps * evalh[1] - evalh[2] - evalh[3];
  const double pd = std::isfinite(lam) ? lam * evalh[0] : evalh[0];
  out[0] = (double)total;
  out[1] = evalh[0];
  out[2] = D + pd;
  out[3] = D;
  return rc;
}

int full_sinkhorn_dev(const double* mu, const double* nu, const double* logmu, const double* lognu, int N,
                      double eps_start, double eps, double lam, int variant, int precision, int maxit,
                      double err, int check_every, double* alpha, double* beta, double* out, double* d_eval,
                      cudaStream_t st, cudaError_t* cerr) {
  if (precision == 2) {
    // float stages while eps >= 64 h^2 (|pot|/eps small enough for float), then double
    const double h = 1.0 / N, e_sw = 64.0 * h * h;
    double o1[4] = {0, 0, 0, 0};
    long long its = 0;
    if (eps_start > e_sw && eps < e_sw) {
      double e_end = e_sw;
      // last float stage is the first eps of the halving sequence below e_sw's bound
      double e = eps_start;
      while (e * 0.5 >= e_sw) e *= 0.5;
      e_end = e;
      int r = full_sinkhorn_impl<float>(mu, nu, logmu, lognu, N, eps_start, e_end, lam, variant, maxit, err,
                                        check_every, alpha, beta, o1, d_eval, st, cerr);
      if (r < 0) return r;
      its += (long long)o1[0];
      int r2 = full_sinkhorn_impl<double>(mu, nu, logmu, lognu, N, 0.5 * e_end, eps, lam, variant, maxit, err,
                                          check_every, alpha, beta, out, d_eval, st, cerr, true);
      out[0] += (double)its;
      return r2;
    }
    precision = eps < e_sw ? 1 : 0;
    if (precision)   // mixed: the double stages take float exponentials of double exponents
      return full_sinkhorn_impl<double>(mu, nu, logmu, lognu, N, eps_start, eps, lam, variant, maxit, err,
                                        check_every, alpha, beta, out, d_eval, st, cerr, true);
  }
  if (precision)
    return full_sinkhorn_impl<double>(mu, nu, logmu, lognu, N, eps_start, eps, lam, variant, maxit, err,
                                      check_every, alpha, beta, out, d_eval, st, cerr);
  return full_sinkhorn_impl<float>(mu, nu, logmu, lognu, N, eps_start, eps, lam, variant, maxit, err,
                                   check_every, alpha, beta, out, d_eval, st, cerr);
}

// ------------------------------------------------------------------------
// Allocation-free variant of the global Sinkhorn.
//
// Some callers cannot allocate device memory while they run this solver: a
// process that has handed all device memory to its own pool at start-up (a
// cudaMalloc would fail or fragment that pool), or a latency-sensitive loop
// that must not pay the implicit device-wide synchronisation of
// cudaMalloc/cudaFree.  For them the working arrays live in one file-scope
// device array of fixed size, reserved on every GPU that loads the library
// for the life of the process.
namespace {
constexpr int kNoAllocMaxN2 = 256 * 256;  // largest grid: N*N <= 65536 (N <= 256)
// log mu, log nu (N*N doubles each), five N*N work arrays of the log-sum-exp
// (double-sized slots, also used for float), one N*N double slot holding two
// float shadow arrays, 8 doubles of reductions and the input-status word.
constexpr long long kNoAllocDoubles = 8LL * kNoAllocMaxN2 + 16;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of the scratch array in the current device's context (host
// code must not use the symbol itself: it is only a host-side stand-in).  It
// is looked up on every call (no allocation, no cache), so it stays right
// after a cudaDeviceReset or under another context of the same device.
cudaError_t noalloc_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// True if p is device (or managed) memory that the current device can use
// directly; host memory, pinned or pageable, is rejected.
bool is_current_device_ptr(const void* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

template <typename R>
int full_sinkhorn_noalloc_impl(const double* mu, const double* nu, const double* logmu, const double* lognu,
                               int N, double eps_start, double eps, double lam, int variant, int maxit,
                               double err, int check_every, double* alpha, double* beta, double* out,
                               double* work, double* d_eval, cudaStream_t st, cudaError_t* cerr) {
  const int n = N * N;
  const double h = 1.0 / N;
  // five work arrays in double-sized slots (float arrays use the first half of each)
  R* in2 = reinterpret_cast<R*>(work);
  R* tmp = reinterpret_cast<R*>(work + n);
  R* w2 = reinterpret_cast<R*>(work + 2 * (long long)n);
  R* z2 = reinterpret_cast<R*>(work + 3 * (long long)n);
  R* tmpz = reinterpret_cast<R*>(work + 4 * (long long)n);
  float* in2f = reinterpret_cast<float*>(work + 5 * (long long)n);
  float* tmpf = in2f + n;
  const int grid = (n + 255) / 256;
  double evalh[6];
  long long total = 0;
  int rc = 0;
  if (check_every < 1) check_every = 1;
  double e = eps_start > eps ? eps_start : eps;
  for (;;) {
    const double kap = std::isfinite(lam) ? e / (1.0 + e / lam) : e;
    const double q = h * h / e;
    k_to_log2<R><<<grid, 256, 0, st>>>(beta, lognu, 1.0 / e, in2, n, in2f);
    lse_all<R>(in2, tmp, w2, N, q, variant, 0, st, in2f, tmpf);
    int it = 0, shift_ok = 0;
    bool conv = false;
    while (it < maxit) {
      k_half<R><<<grid, 256, 0, st>>>(w2, kap, alpha, n);
      k_to_log2<R><<<grid, 256, 0, st>>>(alpha, logmu, 1.0 / e, in2, n, in2f);
      lse_all<R>(in2, tmpz, z2, N, q, variant, shift_ok, st, in2f, tmpf);
      k_half<R><<<grid, 256, 0, st>>>(z2, kap, beta, n);
      k_to_log2<R><<<grid, 256, 0, st>>>(beta, lognu, 1.0 / e, in2, n, in2f);
      lse_all<R>(in2, tmp, w2, N, q, variant, 1, st, in2f, tmpf);
      shift_ok = 1;
      ++it;
      if (it % check_every == 0 || it == maxit) {
        k_sk_eval<R><<<1, 512, 0, st>>>(mu, nu, alpha, beta, w2, nullptr, e, lam, n, d_eval);
        cudaMemcpyAsync(evalh, d_eval, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
        *cerr = cudaStreamSynchronize(st);
        if (*cerr != cudaSuccess) return -1;
        if (err >= 0.0 && evalh[0] <= err * evalh[4]) { conv = true; break; }
        if (!(evalh[0] == evalh[0])) break;
      }
    }
    total += it;
    if (e <= eps) { rc = conv || err < 0.0 ? 0 : 1; break; }
    e = fmax(eps, 0.5 * e);
  }
  k_sk_eval<R><<<1, 512, 0, st>>>(mu, nu, alpha, beta, w2, z2, eps, lam, n, d_eval);
  cudaMemcpyAsync(evalh, d_eval, 6 * sizeof(double), cudaMemcpyDeviceToHost, st);
  *cerr = cudaStreamSynchronize(st);
  if (*cerr != cudaSuccess) return -1;
  const double D = eps * evalh[4] * evalh[5] - eps * evalh[1] - evalh[2] - evalh[3];
  const double pd = std::isfinite(lam) ? lam * evalh[0] : evalh[0];
  out[0] = (double)total;
  out[1] = evalh[0];
  out[2] = D + pd;
  out[3] = D;
  return rc;
}
}  // namespace

cudaError_t launch_prepare_inputs(const double* mu, const double* nu, double* logmu, double* lognu, int n,
                                  int* status, cudaStream_t st);

int domdec_full_sinkhorn_noalloc(const double* mu, const double* nu, int N, double eps_start,
                                            double eps, double lambda, int variant, int precision, int maxit,
                                            double err, int check_every, const double* beta_in, double* alpha,
                                            double* beta, double out[4], void* stream) {
  if (!mu || !nu || !alpha || !beta || !out || N <= 0) return DOMDEC_EINVAL;
  if (!(eps > 0.0) || !(lambda > 0.0) || (variant != 0 && variant != 1) || (precision != 0 && precision != 1) ||
      maxit < 1)
    return DOMDEC_EINVAL;
  if ((long long)N * N > kNoAllocMaxN2) return DOMDEC_ETOOBIG;
  // the kernels read mu, nu, beta_in and write alpha, beta directly: each must be
  // memory of the current device (a host array would fault or, where the GPU can
  // reach host memory, be used silently)
  if (!is_current_device_ptr(mu) || !is_current_device_ptr(nu) || !is_current_device_ptr(alpha) ||
      !is_current_device_ptr(beta) || (beta_in && !is_current_device_ptr(beta_in)))
    return DOMDEC_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) return DOMDEC_ECUDA;
  const int n = N * N;
  double* logmu = base;
  double* lognu = base + n;
  double* work = base + 2 * (long long)n;
  double* d_eval = base + 8LL * kNoAllocMaxN2;
  int* d_status = reinterpret_cast<int*>(d_eval + 8);
  // every call starts from a cleared status word and its own beta
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    if (beta_in) {
      if (beta_in != beta) e = cudaMemcpyAsync(beta, beta_in, n * sizeof(double), cudaMemcpyDefault, st);
    } else {
      e = cudaMemsetAsync(beta, 0, n * sizeof(double), st);
    }
  }
  if (e == cudaSuccess) e = launch_prepare_inputs(mu, nu, logmu, lognu, n, d_status, st);
  int hstat = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return DOMDEC_ECUDA;
  if (hstat) return DOMDEC_EINVAL;
  cudaError_t ce = cudaSuccess;
  int r = precision ? full_sinkhorn_noalloc_impl<double>(mu, nu, logmu, lognu, N, eps_start, eps, lambda,
                                                         variant, maxit, err, check_every, alpha, beta, out,
                                                         work, d_eval, st, &ce)
                    : full_sinkhorn_noalloc_impl<float>(mu, nu, logmu, lognu, N, eps_start, eps, lambda,
                                                        variant, maxit, err, check_every, alpha, beta, out,
                                                        work, d_eval, st, &ce);
  if (r < 0) return DOMDEC_ECUDA;
  return r ? 1 : 0;
}
