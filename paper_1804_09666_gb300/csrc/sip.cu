// sip.cu -- SIP / the Stone method (Veneva & Ayriyan, arXiv:1804.09666, Sec. 2,
// Algorithm 1) with ILU(0) and, optionally, Hotelling-Bodewig band inverses in place
// of the forward/backward substitutions (Remark of Sec. 2; Eq. (1), Appendix).
// One thread per system; FP64.
//
// ILU(0) on the pentadiagonal pattern, row-wise: for k = i-2, i-1 in the pattern,
// l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for j > k in the pattern of row i.  For
// this pattern nothing is dropped, so L (unit; l2 = L[i][i-2], l1 = L[i][i-1]) and
// U (u0 = U[i][i], u1 = U[i][i+1], u2 = U[i][i+2] = e_i) are the exact LU factors.
#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "api_util.h"
#include "kernels.h"
#include "sip_impl.cuh"

namespace band {
namespace {

// Band Hotelling-Bodewig, X_{k+1} = X_k (2I - M X_k), X_0 = diag(M)^{-1}, X kept to
// w diagonals.  Written along a sweep index t (t = i for L, t = n-1-i for U) so that
// both factors look lower triangular: X_j[t] = X[t][t-j], and M's entries along the
// sweep are m0 (diagonal; 1 for L), m1 (one step back), m2 (two steps back).  With
// P = M X:  Pr_j[t] = sum_{o<=min(2,j)} M_o[t] X_{j-o}[t-o], and
//   Xnew_j[t] = 2 X_j[t] - sum_{k=0..j} X_k[t] Pr_{j-k}[t-k].
struct HbArgs {
  Layout L;
  Spill W;
  int w, upper, max_it;
  double tol;
  const double *m0, *m1, *m2;   // L: (nullptr, l1, l2); U: (u0, u1, e-from-input)
  const double* e_in;           // U's second superdiagonal is e itself (input layout)
  double* X[kMaxWidth];         // result
  double* Y[kMaxWidth];         // ping-pong partner
  int32_t* status;
  int32_t* hb_iters;
};

__global__ void __launch_bounds__(64) k_hb(const HbArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (p.status && p.status[s] != BAND_OK) return;
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  const int w = p.w;
  auto row_of = [&](int64_t t) { return p.upper ? n - 1 - t : t; };
  auto Mo = [&](int o, int64_t t) -> double {  // M entry o steps back along the sweep
    const int64_t i = row_of(t);
    const int64_t wi = w0 + i * ws;
    if (o == 0) return p.upper ? p.m0[wi] : 1.0;
    if (o == 1) return p.m1[wi];
    return p.upper ? ldro(p.e_in + q0 + i * es) : p.m2[wi];
  };
  double* const* cur = p.Y;
  double* const* nxt = p.X;
  // X_0 = diag(M)^{-1} into `cur`
  for (int64_t t = 0; t < n; ++t) {
    const int64_t wi = w0 + row_of(t) * ws;
    cur[0][wi] = 1.0 / Mo(0, t);
    for (int j = 1; j < w; ++j) cur[j][wi] = 0.0;
  }
  int it = 0;
  int32_t st = BAND_ERR_NOT_CONVERGED;
  while (it < p.max_it) {
    double xr[3][kMaxWidth];          // X rows t, t-1, t-2 (ring by t % 3)
    double pr[kMaxWidth][kMaxWidth];  // Pr rows t .. t-w+1 (ring by t % w)
    for (int r = 0; r < 3; ++r)
      for (int j = 0; j < kMaxWidth; ++j) xr[r][j] = 0.0;
    for (int r = 0; r < kMaxWidth; ++r)
      for (int j = 0; j < kMaxWidth; ++j) pr[r][j] = 0.0;
    double dmax = 0.0, xmax = 0.0;
    bool nan_seen = false;
    for (int64_t t = 0; t < n; ++t) {
      const int64_t wi = w0 + row_of(t) * ws;
      const int r0 = (int)(t % 3), r1 = (int)((t + 2) % 3), r2 = (int)((t + 1) % 3);
      for (int j = 0; j < w; ++j) xr[r0][j] = cur[j][wi];
      const double mm0 = Mo(0, t);
      const double mm1 = t >= 1 ? Mo(1, t) : 0.0;
      const double mm2 = t >= 2 ? Mo(2, t) : 0.0;
      const int pt = (int)(t % w);
      for (int j = 0; j < w; ++j) {
        double v = mm0 * xr[r0][j];
        if (j >= 1 && t >= 1) v = fma(mm1, xr[r1][j - 1], v);
        if (j >= 2 && t >= 2) v = fma(mm2, xr[r2][j - 2], v);
        pr[pt][j] = v;
      }
      for (int j = 0; j < w; ++j) {
        double acc = 2.0 * xr[r0][j];
        for (int k = 0; k <= j; ++k) {
          if (t - k < 0) break;
          const int pk = (int)((t - k) % w);
          acc = fma(-xr[r0][k], pr[pk][j - k], acc);
        }
        const double old = xr[r0][j];
        nxt[j][wi] = acc;
        const double dd = fabs(acc - old);
        nan_seen |= (acc != acc);
        dmax = fmax(dmax, dd);
        xmax = fmax(xmax, fabs(old));
      }
    }
    ++it;
    double* const* tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (nan_seen || !isfinite(dmax)) { st = BAND_ERR_NONFINITE; break; }
    if (dmax <= p.tol * xmax) { st = BAND_OK; break; }
  }
  // the result must end in X
  if (cur != p.X) {
    for (int64_t t = 0; t < n; ++t) {
      const int64_t wi = w0 + row_of(t) * ws;
      for (int j = 0; j < w; ++j) p.X[j][wi] = cur[j][wi];
    }
  }
  if (p.hb_iters) p.hb_iters[s] = it;
  // a capped HB iteration still gives usable approximate inverses; SIP decides
  if (st == BAND_ERR_NONFINITE) set_status(p.status, s, st);
}

// ---------------------------------------------------------------------------
// SIP with Hotelling-Bodewig inverses, one block per system, the whole system in shared
// memory.  Both halves of the method are row-parallel: an HB iteration computes
// P = M X for every row from the current X, then X <- 2X - X P for every row (each row
// of X_new needs only its own row of X and w rows of P); an SIP update applies the
// banded matrices: r = f - A x, y = L~^{-1} r, x <- x + U~^{-1} y.  The threads of the
// block take rows, the passes are separated by block barriers, and each system stops
// on its own (the block's own reductions), so no system waits for another.  The
// arithmetic and its order per row are those of k_hb / sip_hb, which run the same
// iterations with one thread per system for systems too large for shared memory.
// ---------------------------------------------------------------------------
constexpr int kHbThreads = 256;

struct HbBlockSm {
  double *a, *b, *c, *d, *e, *f;   // n each
  double *XL, *XU;                 // w x n each (diagonal j of row t at j * n + t)
  double *P, *m1, *m2, *m0;        // HB scratch: P (w x n) and M's entries along the sweep
  double *x, *r, *y;               // SIP scratch (over the HB scratch)
};

// Shared-memory doubles per row for width w: A and f, both inverses, and the larger of
// the two scratch sets.
__host__ __device__ inline int64_t hb_block_words_per_row(int w) {
  const int64_t scratch = (w + 3) > 3 ? (w + 3) : 3;
  return 6 + 2 * (int64_t)w + scratch;
}

// One HB inversion in shared memory, sweep coordinates t = 0 .. n-1 (M lower in t):
// X <- X (2I - M X) truncated to w diagonals from X_0 = diag(M)^{-1}.  Returns the
// status for the system (OK, NOT_CONVERGED at the cap: usable, NONFINITE).
template <int W>
__device__ inline int32_t hb_block(const HbBlockSm& S, double* X, int64_t n, int max_it,
                                   double tol, double* red, int* iters) {
  constexpr int w = W;
  for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
    X[t] = 1.0 / S.m0[t];
    for (int j = 1; j < w; ++j) X[j * n + t] = 0.0;
  }
  __syncthreads();
  int it = 0;
  int32_t st = BAND_ERR_NOT_CONVERGED;
  while (it < max_it) {
    // P = M X on the band: P_j[t] = m0 X_j[t] + m1 X_{j-1}[t-1] + m2 X_{j-2}[t-2]
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      const double mm0 = S.m0[t];
      const double mm1 = t >= 1 ? S.m1[t] : 0.0;
      const double mm2 = t >= 2 ? S.m2[t] : 0.0;
      for (int j = 0; j < w; ++j) {
        double v = mm0 * X[j * n + t];
        if (j >= 1 && t >= 1) v = fma(mm1, X[(j - 1) * n + t - 1], v);
        if (j >= 2 && t >= 2) v = fma(mm2, X[(j - 2) * n + t - 2], v);
        S.P[j * n + t] = v;
      }
    }
    __syncthreads();
    // X_new_j[t] = 2 X_j[t] - sum_{k<=j} X_k[t] P_{j-k}[t-k]; a row needs only its own X
    double dmax = 0.0, xmax = 0.0;
    bool nan = false;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
      double xo[W], xn[W];
#pragma unroll
      for (int j = 0; j < w; ++j) xo[j] = X[j * n + t];
#pragma unroll
      for (int j = 0; j < w; ++j) {
        double acc = 2.0 * xo[j];
#pragma unroll
        for (int k = 0; k <= j; ++k) {
          if (t - k < 0) break;
          acc = fma(-xo[k], S.P[(j - k) * n + t - k], acc);
        }
        xn[j] = acc;
        nan |= (acc != acc);
        dmax = fmax(dmax, fabs(acc - xo[j]));
        xmax = fmax(xmax, fabs(xo[j]));
      }
#pragma unroll
      for (int j = 0; j < w; ++j) X[j * n + t] = xn[j];
    }
    const double dm = block_max(nan ? INFINITY : dmax, red);
    const double xm = block_max(xmax, red);
    ++it;
    if (!(dm < INFINITY)) { st = BAND_ERR_NONFINITE; break; }
    if (dm <= tol * xm) { st = BAND_OK; break; }
  }
  __syncthreads();
  *iters = it;
  return st;
}

struct HbBlockArgs {
  int hb_max_it;
  double hb_tol;
  int64_t smem_rows;     // systems with more rows are left to the one-thread path
};

template <int W>
__global__ void __launch_bounds__(kHbThreads) k_sip_hb_block(const SipArgs p, const HbBlockArgs h) {
  extern __shared__ double hb_smem[];
  __shared__ double red[kHbThreads / 32];
  constexpr int w = W;
  for (int64_t s = blockIdx.x; s < p.L.nsys; s += gridDim.x) {
    const int64_t n = p.L.rows(s);
    if (n > h.smem_rows) continue;
    if (p.status && p.status[s] != BAND_OK) {        // ILU(0) met a zero pivot
      if (threadIdx.x == 0) {
        if (p.iters) p.iters[s] = 0;
        if (p.resid) p.resid[s] = NAN;
      }
      continue;
    }
    const int64_t q0 = p.L.base(s), es = p.L.stride();
    const int64_t w0 = p.W.base(s), ws = p.W.stride();
    HbBlockSm S;
    S.a = hb_smem; S.b = S.a + n; S.c = S.b + n; S.d = S.c + n; S.e = S.d + n; S.f = S.e + n;
    S.XL = S.f + n; S.XU = S.XL + w * n;
    S.P = S.XU + w * n; S.m0 = S.P + w * n; S.m1 = S.m0 + n; S.m2 = S.m1 + n;
    S.x = S.P; S.r = S.x + n; S.y = S.r + n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const Row A = load_row(p, q0 + i * es, i, n);
      S.a[i] = A.a; S.b[i] = A.b; S.c[i] = A.c; S.d[i] = A.d; S.e[i] = A.e; S.f[i] = A.f;
      // L along t = i: (1, l1, l2)
      S.m0[i] = 1.0;
      S.m1[i] = p.l1[w0 + i * ws];
      S.m2[i] = p.l2[w0 + i * ws];
    }
    __syncthreads();
    int itl = 0, itu = 0;
    const int32_t stl = hb_block<W>(S, S.XL, n, h.hb_max_it, h.hb_tol, red, &itl);
    // U along t = n-1-i: (u0, u1, e)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t t = n - 1 - i;
      S.m0[t] = p.u0[w0 + i * ws];
      S.m1[t] = p.u1[w0 + i * ws];
      S.m2[t] = S.e[i];
    }
    __syncthreads();
    const int32_t stu = hb_block<W>(S, S.XU, n, h.hb_max_it, h.hb_tol, red, &itu);
    if (stl == BAND_ERR_NONFINITE || stu == BAND_ERR_NONFINITE) {
      if (threadIdx.x == 0) {
        if (p.iters) p.iters[s] = 0;
        if (p.resid) p.resid[s] = NAN;
        set_status(p.status, s, BAND_ERR_NONFINITE);
      }
      __syncthreads();
      continue;
    }
    // SIP in correction form from x^0 = 0
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) S.x[i] = 0.0;
    __syncthreads();
    int k = 0;
    double rn = 0.0;
    int32_t st = BAND_ERR_NOT_CONVERGED;
    for (;;) {
      double loc = 0.0;
      bool nan = false;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double xm2 = i >= 2 ? S.x[i - 2] : 0.0, xm1 = i >= 1 ? S.x[i - 1] : 0.0;
        const double xp1 = i + 1 < n ? S.x[i + 1] : 0.0, xp2 = i + 2 < n ? S.x[i + 2] : 0.0;
        double ax = S.c[i] * S.x[i];
        ax = fma(S.a[i], xm2, ax);
        ax = fma(S.b[i], xm1, ax);
        ax = fma(S.d[i], xp1, ax);
        ax = fma(S.e[i], xp2, ax);
        const double r = S.f[i] - ax;
        S.r[i] = r;
        nan |= (r != r);
        loc = fmax(loc, fabs(r));
      }
      rn = block_max(nan ? INFINITY : loc, red);     // ends with a barrier: r complete
      if (!(rn < INFINITY)) { rn = NAN; st = BAND_ERR_NONFINITE; break; }
      if (rn < p.tol) { st = BAND_OK; break; }
      if (k >= p.max_it) break;
      // y = L~^{-1} r (lower band along t = i)
      for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        double yv = 0.0;
#pragma unroll
        for (int j = 0; j < w; ++j)
          if (t - j >= 0) yv = fma(S.XL[j * n + t], S.r[t - j], yv);
        S.y[t] = yv;
      }
      __syncthreads();
      // x += U~^{-1} y (row i of U~^{-1} is row t = n-1-i of X_U: entries at i .. i+w-1)
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t t = n - 1 - i;
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < w; ++j)
          if (i + j < n) acc = fma(S.XU[j * n + t], S.y[i + j], acc);
        S.x[i] = S.x[i] + acc;
      }
      __syncthreads();
      ++k;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p.x[q0 + i * es] = S.x[i];
    if (threadIdx.x == 0) {
      if (p.iters) p.iters[s] = k;
      if (p.resid) p.resid[s] = rn;
      set_status(p.status, s, st);
    }
    __syncthreads();
  }
}

template <int W>
cudaError_t launch_hb_w(const SipArgs& sa, const HbBlockArgs& h, size_t smem, int64_t nsys,
                        cudaStream_t st) {
  const cudaError_t e = tail_prepare((const void*)k_sip_hb_block<W>);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // as many blocks as fit on the SMs at once (227 KiB of shared memory per SM)
  const int64_t per_sm = std::max<int64_t>(1, (int64_t)(227 << 10) / (int64_t)(smem + 1024));
  int64_t grid = (int64_t)(nsm > 0 ? nsm : 1) * per_sm;
  if (grid > nsys) grid = nsys;
  k_sip_hb_block<W><<<(unsigned)grid, kHbThreads, smem, st>>>(sa, h);
  return cudaGetLastError();
}

cudaError_t launch_sip_hb_block(const SipArgs& sa, int width, int hb_max_it, double hb_tol,
                                size_t smem, int64_t nsys, cudaStream_t st) {
  HbBlockArgs h{hb_max_it, hb_tol, (int64_t)(smem / ((size_t)hb_block_words_per_row(width) * sizeof(double)))};
  switch (width) {
    case 1: return launch_hb_w<1>(sa, h, smem, nsys, st);
    case 2: return launch_hb_w<2>(sa, h, smem, nsys, st);
    case 3: return launch_hb_w<3>(sa, h, smem, nsys, st);
    case 4: return launch_hb_w<4>(sa, h, smem, nsys, st);
    case 5: return launch_hb_w<5>(sa, h, smem, nsys, st);
    case 6: return launch_hb_w<6>(sa, h, smem, nsys, st);
    case 7: return launch_hb_w<7>(sa, h, smem, nsys, st);
    default: return launch_hb_w<8>(sa, h, smem, nsys, st);
  }
}

// Algorithm 1 with exact substitutions, first update on the two-sided schedule: 16
// systems per warp (lanes l, l ^ 16).
__global__ void __launch_bounds__(128) k_sip_two(const SipArgs p) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t t = warp * 16 + (threadIdx.x & 15);
  sip_two_sided(p, t, t < p.L.nsys);
}

__global__ void __launch_bounds__(256, 4) k_sip_resid(const SipArgs p) {
  sip_resid_cell(p, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_sip_decide(const SipArgs p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p.L.nsys) sip_decide_one(p, t);
}

__global__ void __launch_bounds__(128) k_ilu0(const SipArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  set_status(p.status, s, ilu0_into(p, s) ? BAND_OK : BAND_ERR_ZERO_PIVOT);
}

__global__ void __launch_bounds__(128) k_sip(const SipArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (p.w == 0) {            // ILU(0) is fused into the first update
    sip_literal(p, s, nullptr);
    return;
  }
  if (p.status && p.status[s] != BAND_OK) {  // ILU(0) or HB failed for this system
    if (p.iters) p.iters[s] = 0;
    if (p.resid) p.resid[s] = NAN;
    return;
  }
  sip_hb(p, s);
}

}  // namespace

SipWs carve_sip(const band_desc* d, int32_t width, void* base, size_t* bytes) {
  Carve c(base);
  SipWs w{};
  const size_t rows = (size_t)spill_rows(d) * sizeof(double);
  w.l2 = (double*)c.take(rows);
  w.l1 = (double*)c.take(rows);
  w.u0 = (double*)c.take(rows);
  w.ru0 = (double*)c.take(rows);
  w.u1 = (double*)c.take(rows);
  w.y = (double*)c.take(rows);
  w.xb = (double*)c.take(rows);
  for (int j = 0; j < 2 * width; ++j) w.X[j] = (double*)c.take(rows);
  for (int j = 0; j < 2 * width; ++j) w.T[j] = (double*)c.take(rows);
  const size_t ns = (size_t)(d->nsys > 0 ? d->nsys : 1);
  w.st = (int32_t*)c.take(sizeof(int32_t) * ns);
  w.tail_count = (unsigned long long*)c.take(sizeof(unsigned long long));
  w.tail_list = (int64_t*)c.take(sizeof(int64_t) * ns);
  w.tail_rn = (double*)c.take(sizeof(double) * ns);
  w.rn_sys = (unsigned long long*)c.take(sizeof(unsigned long long) * ns);
  w.pend = (int32_t*)c.take(sizeof(int32_t) * ns);
  *bytes = c.size();
  return w;
}

size_t sip_workspace_bytes(const band_desc* d, int32_t width) {
  if (width < 0 || width > kMaxWidth) return 0;
  size_t b = 0;
  carve_sip(d, width, nullptr, &b);
  return b;
}

}  // namespace band

using namespace band;

namespace band {

__global__ void __launch_bounds__(kTailThreads) k_sip_tail(const SipArgs p, int64_t smem_rows) {
  __shared__ Aff sh[kTailThreads];
  __shared__ double red[kTailThreads / 32];
  extern __shared__ double tail_smem[];
  const unsigned long long count = *p.tail_count;
  for (unsigned long long it = blockIdx.x; it < count; it += gridDim.x) {
    const int64_t s = p.tail_list[it];
    sip_tail_block(p, s, p.tail_rn[it], sh, red, tail_smem, smem_rows);
  }
}

// Dynamic shared memory of a tail launch for systems of at most n_max rows: the whole
// system when it fits in kTailSmemMax bytes, else the largest copy that fits (smaller
// systems of a ragged batch still use it).  One block per SM either way.
size_t tail_smem_bytes(int64_t n_max) {
  const size_t want = (size_t)n_max * sizeof(double) * kTailSmemArrays;
  return want < kTailSmemMax ? want : kTailSmemMax;
}

// Opt a tail kernel in to kTailSmemMax bytes of dynamic shared memory, once per kernel
// and device (the first call normally comes before any graph capture).
cudaError_t tail_prepare(const void* kernel) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& kd : done)
    if (kd.first == kernel && kd.second == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax);
  if (e == cudaSuccess) done.emplace_back(kernel, dev);
  return e;
}

cudaError_t launch_sip_tail(const SipArgs& p, int64_t nsys, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = nsm > 0 ? nsm : 1;
  if (blocks > nsys) blocks = nsys;
  if (blocks < 1) blocks = 1;
  const cudaError_t e = tail_prepare((const void*)k_sip_tail);
  if (e != cudaSuccess) return e;
  const size_t smem = tail_smem_bytes(p.L.n);
  k_sip_tail<<<(unsigned)blocks, kTailThreads, smem, st>>>(p, tail_smem_rows(smem));
  return cudaGetLastError();
}

band_status make_sip(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                     double tol, int32_t max_it, int32_t width, int32_t* iters, double* resid,
                     int32_t* sys_status, void* ws, size_t ws_bytes, SipArgs* sa, SipWs* wout) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64 || desc->schedule == BAND_SCHED_GRID)
    return BAND_ERR_ARG;
  if (width < 0 || width > kMaxWidth || max_it < 0) return BAND_ERR_ARG;
  // id lists: Algorithm 1 with exact substitutions only, statuses indexed by id
  if (desc->systems && (width != 0 || !sys_status)) return BAND_ERR_ARG;
  if (!(tol >= 0.0)) return BAND_ERR_ARG;
  // TD systems are treated as PD with a = e = 0; that needs a and e arrays.
  if (!diag || !f || !x || !diag[0] || !diag[1] || !diag[2] || !diag[3] || !diag[4])
    return BAND_ERR_ARG;
  if (!arrays_aligned(BAND_F64, diag, f, x, sys_status) || !aligned_all(8, {resid}) ||
      !aligned_all(4, {iters}))
    return BAND_ERR_ARG;
  size_t need = 0;
  carve_sip(desc, width, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const SipWs w = carve_sip(desc, width, ws, &need);
  *sa = SipArgs{};
  sa->L = layout_of(desc);
  sa->W = spill_of(desc);
  sa->a = (const double*)diag[0]; sa->b = (const double*)diag[1]; sa->c = (const double*)diag[2];
  sa->d = (const double*)diag[3]; sa->e = (const double*)diag[4];
  sa->f = (const double*)f;
  sa->x = (double*)x;
  sa->xb = w.xb;
  sa->y = w.y;
  sa->l2 = w.l2; sa->l1 = w.l1; sa->u0 = w.u0; sa->ru0 = w.ru0; sa->u1 = w.u1;
  sa->w = width;
  sa->tol = tol;
  sa->max_it = max_it;
  sa->iters = iters;
  sa->status = sys_status ? sys_status : w.st;
  sa->resid = resid;
  if (width == 0) {
    sa->tail_count = w.tail_count;
    sa->tail_list = w.tail_list;
    sa->tail_rn = w.tail_rn;
    sa->pend = w.pend;
    sa->rn_sys = w.rn_sys;
    // Algorithm 1's first update may run on the two-sided schedule (band_schedule)
    sa->two_sided = choose_two_sided(desc, false) ? 1 : 0;
  }
  if (wout) *wout = w;
  return BAND_OK;
}

}  // namespace band

extern "C" band_status band_sip(const band_desc* desc, const void* const diag[5], const void* f,
                                void* x, double tol, int32_t max_it, int32_t width,
                                int32_t hb_max_it, double hb_tol, int32_t* iters, double* resid,
                                int32_t* sys_status, void* ws, size_t ws_bytes, void* stream) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64 || desc->schedule == BAND_SCHED_GRID)
    return BAND_ERR_ARG;
  if (width < 0 || width > kMaxWidth || max_it < 0 || hb_max_it < 0) return BAND_ERR_ARG;
  if (!(tol >= 0.0) || !(hb_tol >= 0.0)) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  SipArgs sa;
  SipWs w;
  const band_status v = make_sip(desc, diag, f, x, tol, max_it, width, iters, resid, sys_status,
                                 ws, ws_bytes, &sa, &w);
  if (v != BAND_OK) return v;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned g128 = (unsigned)((desc->nsys + 127) / 128);
  const unsigned g64 = (unsigned)((desc->nsys + 63) / 64);
  if (width > 0) {
    k_ilu0<<<g128, 128, 0, st>>>(sa);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    // systems that fit in shared memory: one block each, row-parallel
    const size_t per_row = (size_t)hb_block_words_per_row(width) * sizeof(double);
    if ((size_t)desc->n * per_row <= kTailSmemMax) {
      const cudaError_t e = launch_sip_hb_block(sa, width, hb_max_it, hb_tol,
                                                (size_t)desc->n * per_row, desc->nsys, st);
      return cuda_status(e);
    }
    for (int upper = 0; upper < 2; ++upper) {
      HbArgs h{};
      h.L = sa.L;
      h.W = sa.W;
      h.w = width;
      h.upper = upper;
      h.max_it = hb_max_it;
      h.tol = hb_tol;
      h.m0 = upper ? w.u0 : nullptr;
      h.m1 = upper ? w.u1 : w.l1;
      h.m2 = upper ? nullptr : w.l2;
      h.e_in = sa.e;
      for (int j = 0; j < width; ++j) {
        h.X[j] = w.X[upper * width + j];
        h.Y[j] = w.T[upper * width + j];
      }
      h.status = sa.status;
      h.hb_iters = nullptr;
      k_hb<<<g64, 64, 0, st>>>(h);
      if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    }
    for (int j = 0; j < width; ++j) {
      sa.XL[j] = w.X[j];
      sa.XU[j] = w.X[width + j];
    }
  }
  if (width == 0 &&
      (cudaMemsetAsync(sa.tail_count, 0, sizeof(unsigned long long), st) != cudaSuccess ||
       cudaMemsetAsync(sa.rn_sys, 0, (size_t)((char*)(sa.pend + desc->nsys) - (char*)sa.rn_sys),
                       st) != cudaSuccess))
    return BAND_ERR_CUDA;
  if (sa.two_sided) {
    const int64_t threads = (desc->nsys + 15) / 16 * 32;
    k_sip_two<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(sa);
  } else {
    k_sip<<<g128, 128, 0, st>>>(sa);
  }
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  if (width == 0) {
    k_sip_resid<<<(unsigned)((resid_cells(sa.L) + 255) / 256), 256, 0, st>>>(sa);
    k_sip_decide<<<(unsigned)((desc->nsys + 255) / 256), 256, 0, st>>>(sa);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    return cuda_status(launch_sip_tail(sa, desc->nsys, st));
  }
  return BAND_OK;
}
