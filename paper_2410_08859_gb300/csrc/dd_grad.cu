// Adjoint of the unbalanced OT value: gradients of
//   S(mu, nu, x) = max_{alpha, beta} D(alpha, beta)      (Eq. dual-problem, nu_- = 0, D_i = lam KL)
// with respect to the weights mu, nu and the source positions x, from dual
// potentials (alpha, beta).  The paper does not differentiate S; by the
// envelope theorem the derivatives of S at the optimum are those of D at fixed
// potentials:
//   dS/dmu(x) = eps |nu| - eps P_X(x)/mu(x) - lam (e^{-alpha(x)/lam} - 1)
//   dS/dnu(y) = eps |mu| - eps P_Y(y)/nu(y) - lam (e^{-beta(y)/lam} - 1)
//   dS/dx     = 2 P_X(x) (x - T(x)),   T(x) = sum_y pi(x,y) y / P_X(x)
// with pi = exp((alpha + beta - c)/eps) mu x nu, c = |x - y|^2 on the grid
// {0..N-1}^2 / N (row-major, x = i N + j has coordinates (i, j) / N).  For
// lam = infinity the penalty terms become alpha and beta.
//
// The plan is never formed.  |x - y|^2 = h^2 ((i-k)^2 + (j-l)^2) makes every
// sum over y separable: a pass along grid rows (over l) and one along columns
// (over k).  The barycentric displacement T(x) - x is carried through the
// passes as conditional means (bounded by the grid size, no cancellation
// against |x|):
//   pass 1  a(k, j)  = log2 sum_l 2^{f(k,l) - Q (j-l)^2}
//           m(k, j)  = sum_l w (l - j) / sum_l w            (w: the summed terms)
//   pass 2  L(i, j)  = log2 sum_k 2^{a(k,j) - Q (i-k)^2}
//           M1(i, j) = sum_k w (k - i) / sum_k w,  M2(i, j) = sum_k w m(k, j) / sum_k w
// with f = (beta/eps + log nu) log2 e and Q = h^2/eps log2 e; then
// P_X = mu exp(alpha/eps + L ln 2) and T(x) - x = h (M1, M2).  The Y side is
// the same without moments, with f = (alpha/eps + log mu) log2 e.
//
// Terms more than 2^-cut below the running maximum are skipped after a float
// test on shadow values (as in the separable Sinkhorn).  f and the pass-1 sums
// are kept in double: at eps = (2/N)^2 they reach ~1e4 in log2 units, where a
// float carries only ~1e-3 absolute.  Each surviving term's exponent
// f - Q d^2 - max is formed in double (three operations) and only the
// exponential and the sums run in R: float (ex2.approx) or double.
#include <cmath>

#include "dd_common.cuh"
#include "domdec.h"

namespace {

template <typename R> __device__ __forceinline__ float adj_cut() { return sizeof(R) == 4 ? 33.0f : 65.0f; }
__device__ __forceinline__ float adj_ex2(float v) { return dd_ex2(v); }
__device__ __forceinline__ double adj_ex2(double v) { return dd_ex2(v); }

// One windowed 1-D log-sum-exp per target with P lanes, plus K conditional
// means: mom(m, e, acc) adds e * g_k(m) to acc[k]; out[k] receives mean k.
// Returns the log2-sum in double; src(m) is double, srcf(m) its float shadow.
template <typename R, int K, typename FS, typename FF, typename FM>
__device__ __forceinline__ double lse_moments(FS src, FF srcf, FM mom, int M, int ctr, float Qf, double Qd,
                                              int part, int P, R* out) {
  float mxf = -INFINITY;
  for (int m = part; m < M; m += P) {
    float d = (float)(ctr - m);
    mxf = fmaxf(mxf, srcf(m) - Qf * d * d);
  }
  for (int o = 1; o < P; o <<= 1) mxf = fmaxf(mxf, __shfl_xor_sync(0xffffffffu, mxf, o));
  const bool any = mxf > -INFINITY;
  const float cut = adj_cut<R>();
  const double mx = any ? double(mxf) : 0.0;
  R acc = R(0);
  R acm[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < (K > 0 ? K : 1); ++k) acm[k] = R(0);
  if (any) {
    for (int m = part; m < M; m += P) {
      float d = (float)(ctr - m);
      if (srcf(m) - Qf * d * d - mxf > -cut) {
        const double dr = double(ctr - m);
        R e = adj_ex2(R(src(m) - Qd * dr * dr - mx));
        acc += e;
        if constexpr (K > 0) mom(m, e, acm);
      }
    }
  }
  for (int o = 1; o < P; o <<= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
#pragma unroll
    for (int k = 0; k < K; ++k) acm[k] += __shfl_xor_sync(0xffffffffu, acm[k], o);
  }
  if (!any || !(acc > R(0))) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = R(0);
    return -INFINITY;
  }
  const R inv = R(1) / acc;
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = acm[k] * inv;
  return mx + (double)dd_lg2(acc);
}

constexpr int kAdjLanes = 4;  // lanes per target

template <typename R>
struct AdjBufs {
  const double* in;  // f (log2 units), N*N
  const float* inf;  // float shadow of f
  double* a;         // pass-1 log2-sums
  float* af;         // float shadow of a
  R* m;              // pass-1 conditional means (X side only)
};

// Pass 1 (block = grid row k): a[k, j], and m[k, j] when MOM.
template <typename R, bool MOM>
__global__ void __launch_bounds__(1024) k_adj_rows(AdjBufs<R> B, int N, double Q) {
  extern __shared__ __align__(16) unsigned char sm[];
  double* row = reinterpret_cast<double*>(sm);
  float* rowf = reinterpret_cast<float*>(row + N);
  const int k = blockIdx.x;
  for (int l = threadIdx.x; l < N; l += blockDim.x) {
    row[l] = B.in[(long long)k * N + l];
    rowf[l] = B.inf[(long long)k * N + l];
  }
  __syncthreads();
  const float Qf = (float)Q;
  const int P = kAdjLanes, nt = (N * P + 31) & ~31;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int j0 = t / P, part = t % P, j = min(j0, N - 1);
    R mo[1];
    double v = lse_moments<R, MOM ? 1 : 0>(
        [&](int l) { return row[l]; }, [&](int l) { return rowf[l]; },
        [&](int l, R e, R* acc) { acc[0] += e * R(l - j); }, N, j, Qf, Q, part, P, mo);
    if (part == 0 && j0 < N) {
      const long long o = (long long)k * N + j;
      B.a[o] = v;
      B.af[o] = (float)v;
      if (MOM) B.m[o] = mo[0];
    }
  }
}

struct AdjOut {
  const double* mu;     // weights of the side being differentiated (mu for the X side, nu for the Y side)
  const double* pot;    // its potential (alpha for the X side, beta for the Y side)
  double* grad;         // d S / d weight
  double* grad_x;       // X side: d S / d x (2 per point), may be NULL
  double* marg;         // plan marginal of this side (N*N scratch, for the value)
  const double* sums;   // [|mu|, |nu|]
  int side;             // 0: X side, 1: Y side
  double eps, lam, h;
};

// Pass 2 (block = (column tile, grid row i)) and the gradient epilogue.
template <typename R, bool MOM>
__global__ void __launch_bounds__(256) k_adj_cols(AdjBufs<R> B, AdjOut O, int N, double Q) {
  const int P = kAdjLanes;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = t / P, part = t % P, j = min(j0, N - 1);
  const int i = blockIdx.y;
  const double* col = B.a + j;
  const float* colf = B.af + j;
  const R* colm = MOM ? B.m + j : nullptr;
  R mo[2];
  double L = lse_moments<R, MOM ? 2 : 0>(
      [&](int k) { return col[(long long)k * N]; }, [&](int k) { return colf[(long long)k * N]; },
      [&](int k, R e, R* acc) {
        acc[0] += e * R(k - i);
        acc[1] += e * colm[(long long)k * N];
      },
      N, i, (float)Q, Q, part, P, mo);
  if (part != 0 || j0 >= N) return;
  const long long x = (long long)i * N + j;
  const double eps = O.eps, lam = O.lam;
  const double pot = O.pot[x], w = O.mu[x];
  // P(x)/w(x) = exp(pot/eps + L ln 2)
  const double ratio = exp(pot / eps + L * DD_LN2);
  const double marg = w * ratio;
  O.marg[x] = marg;
  const double other = O.sums[O.side == 0 ? 1 : 0];
  const double pen = isfinite(lam) ? -lam * (exp(-pot / lam) - 1.0) : pot;
  O.grad[x] = eps * other - eps * ratio + pen;
  if (MOM && O.grad_x) {
    O.grad_x[2 * x] = -2.0 * marg * O.h * (double)mo[0];
    O.grad_x[2 * x + 1] = -2.0 * marg * O.h * (double)mo[1];
  }
}

// f = (pot/eps + log w) log2 e and its float shadow; marks a non-positive or
// non-finite weight or a non-finite potential in *bad.
__global__ void k_adj_prep(const double* __restrict__ pot, const double* __restrict__ w, double inv_eps,
                           double* __restrict__ f, float* __restrict__ fs, int n, int* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double wi = w[i], pi = pot[i];
    if (!(wi > 0.0) || !isfinite(wi) || !isfinite(pi)) atomicOr(bad, 1);
    const double v = (pi * inv_eps + log(wi)) * DD_LOG2E;
    f[i] = v;
    fs[i] = (float)v;
  }
}

// Block partials of [|mu|, |nu|] (grid-stride; summed by k_sum_partials).
__global__ void __launch_bounds__(512) k_adj_masses(const double* mu, const double* nu, int n, double* partials) {
  __shared__ double red[33 * 2];
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[0] += mu[i];
    v[1] += nu[i];
  }
  block_sum_to<2>(v, red, partials);
}

// Block partials of [|P_X pi|, |P_Y pi|, sum lam (e^{-alpha/lam} - 1) mu, sum lam (e^{-beta/lam} - 1) nu].
__global__ void __launch_bounds__(512)
k_adj_value(const double* mu, const double* nu, const double* alpha, const double* beta, const double* px,
            const double* py, double lam, int n, double* partials) {
  __shared__ double red[33 * 4];
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  const bool fin = isfinite(lam);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    v[0] += px[i];
    v[1] += py[i];
    v[2] += fin ? lam * (exp(-alpha[i] / lam) - 1.0) * mu[i] : -alpha[i] * mu[i];
    v[3] += fin ? lam * (exp(-beta[i] / lam) - 1.0) * nu[i] : -beta[i] * nu[i];
  }
  block_sum_to<4>(v, red, partials);
}

// out = [D(alpha, beta), |mu|, |nu|, |P_X pi|, |P_Y pi|] from sums = [|mu|, |nu|] and
// vsum = k_adj_value's totals.
__global__ void k_adj_finish(const double* sums, const double* vsum, double eps, double* out) {
  if (threadIdx.x != 0) return;
  out[0] = eps * sums[0] * sums[1] - eps * vsum[0] - vsum[2] - vsum[3];
  out[1] = sums[0];
  out[2] = sums[1];
  out[3] = vsum[0];
  out[4] = vsum[1];
}

// Scratch (device): px, py, sums (+ value totals), block partials; f, a (double)
// and their float shadows; m in R.
template <typename R>
cudaError_t adjoint_impl(const double* mu, const double* nu, const double* alpha, const double* beta, int N,
                         double eps, double lam, double* grad_mu, double* grad_nu, double* grad_x, double* d_out,
                         unsigned char* scratch, int* d_bad, cudaStream_t st) {
  const long long n = (long long)N * N;
  unsigned char* p = scratch;
  auto take = [&](size_t bytes) {
    unsigned char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  double* px = reinterpret_cast<double*>(take(n * sizeof(double)));
  double* py = reinterpret_cast<double*>(take(n * sizeof(double)));
  double* sums = reinterpret_cast<double*>(take(8 * sizeof(double)));  // [0..1] masses, [4..7] value totals
  double* partials = reinterpret_cast<double*>(take(kRedBlocks * 4 * sizeof(double)));
  double* f = reinterpret_cast<double*>(take(n * sizeof(double)));
  double* a = reinterpret_cast<double*>(take(n * sizeof(double)));
  R* m = reinterpret_cast<R*>(take(n * sizeof(R)));
  float* fs = reinterpret_cast<float*>(take(n * sizeof(float)));
  float* as = reinterpret_cast<float*>(take(n * sizeof(float)));

  const double h = 1.0 / N, Q = h * h / eps * DD_LOG2E;
  const int eb = (int)std::min<long long>((n + 255) / 256, 4096);
  const int thr_rows = std::min(1024, ((N * kAdjLanes + 31) / 32) * 32);
  const size_t smem_rows = (size_t)N * (sizeof(double) + sizeof(float));
  const dim3 gcols((N * kAdjLanes + 255) / 256, N);
  AdjBufs<R> B{f, fs, a, as, m};

  const int G = red_blocks(n, 512, partials);
  k_adj_masses<<<G, 512, 0, st>>>(mu, nu, (int)n, partials);
  k_sum_partials<<<1, 32, 0, st>>>(partials, G, 2, sums);
  // X side: f = beta/eps + log nu summed over y for every x, with moments.
  k_adj_prep<<<eb, 256, 0, st>>>(beta, nu, 1.0 / eps, f, fs, (int)n, d_bad);
  k_adj_rows<R, true><<<N, thr_rows, smem_rows, st>>>(B, N, Q);
  AdjOut OX{mu, alpha, grad_mu, grad_x, px, sums, 0, eps, lam, h};
  k_adj_cols<R, true><<<gcols, 256, 0, st>>>(B, OX, N, Q);
  // Y side: f = alpha/eps + log mu summed over x for every y.
  k_adj_prep<<<eb, 256, 0, st>>>(alpha, mu, 1.0 / eps, f, fs, (int)n, d_bad);
  k_adj_rows<R, false><<<N, thr_rows, smem_rows, st>>>(B, N, Q);
  AdjOut OY{nu, beta, grad_nu, nullptr, py, sums, 1, eps, lam, h};
  k_adj_cols<R, false><<<gcols, 256, 0, st>>>(B, OY, N, Q);
  k_adj_value<<<G, 512, 0, st>>>(mu, nu, alpha, beta, px, py, lam, (int)n, partials);
  k_sum_partials<<<1, 32, 0, st>>>(partials, G, 4, sums + 4);
  k_adj_finish<<<1, 32, 0, st>>>(sums, sums + 4, eps, d_out);
  return cudaGetLastError();
}

template <typename R>
size_t adjoint_scratch_bytes(int N) {
  const size_t n = (size_t)N * N;
  auto r = [](size_t b) { return (b + 255) & ~size_t(255); };
  return 4 * r(n * 8) + r(64) + r(kRedBlocks * 4 * 8) + r(n * sizeof(R)) + 2 * r(n * 4);
}

}  // namespace

// Device entry used by the C ABI: all pointers device, scratch from
// adjoint_scratch_size.  d_out receives 5 doubles; *d_bad is or-ed with 1 on
// invalid inputs.
size_t adjoint_scratch_size(int N, int precision) {
  return precision == DOMDEC_FP32 ? adjoint_scratch_bytes<float>(N) : adjoint_scratch_bytes<double>(N);
}

cudaError_t adjoint_dev(const double* mu, const double* nu, const double* alpha, const double* beta, int N,
                        double eps, double lam, int precision, double* grad_mu, double* grad_nu, double* grad_x,
                        double* d_out, void* scratch, int* d_bad, cudaStream_t st) {
  if (N > 4096) return cudaErrorInvalidValue;  // shared row of pass 1: 12 N bytes
  unsigned char* s = static_cast<unsigned char*>(scratch);
  if (precision == DOMDEC_FP32)
    return adjoint_impl<float>(mu, nu, alpha, beta, N, eps, lam, grad_mu, grad_nu, grad_x, d_out, s, d_bad, st);
  return adjoint_impl<double>(mu, nu, alpha, beta, N, eps, lam, grad_mu, grad_nu, grad_x, d_out, s, d_bad, st);
}
