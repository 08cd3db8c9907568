// sip2d.cu -- band_sip2d: Stone's method (Sec. 2, Algorithm 1) on a batch of
// two-dimensional five-point systems, the setting where ILU(0) is incomplete.
//
// Unknown k = y nx + x of an nx x ny grid; row k holds s_k (column k - nx), w_k (k - 1),
// c_k (k), e_k (k + 1), t_k (k + nx), stored in the a, b, c, d, e slots of the band
// arrays; entries that would leave the grid are read but never used.  ILU(0) keeps L's
// and U's entries on A's pattern (L unit lower with ls, lw; U with uc and A's own e, t):
//   ls_k = s_k / uc_{k-nx},  lw_k = w_k / uc_{k-1},  uc_k = c_k - ls_k t_{k-nx} - lw_k e_{k-1};
// the fill products ls_k e_{k-nx} (column k - nx + 1) and lw_k t_{k-1} (column k + nx - 1)
// are dropped, so K = LU - A lives on those two diagonals.  Algorithm 1 from x^0 = 0:
// while max|f - A x| >= tol, solve L y = K x + f (forward), U x = y (backward).
// One thread per system runs the factorisation and every update: three sequential
// passes per update over the system's rows (residual, forward, backward) on interleaved
// data (coalesced across the warp's systems); the neighbours k - 1 and k + 1 are kept in
// registers, those at k -+ nx re-read (the thread wrote them nx rows before: L1 / L2).
// Statuses: OK, NOT_CONVERGED (max_it updates), ZERO_PIVOT (uc_k = 0), NONFINITE.
#include <cstdint>

#include "api_util.h"
#include "kernels.h"

namespace band {

namespace {

struct Sip2dArgs {
  Layout L;
  Spill W;
  int64_t nx, ny;
  const double *s, *w, *c, *e, *t, *f;
  double* x;
  double *ls, *lw, *ruc, *y;
  double tol;
  int32_t max_it;
  int32_t* iters;
  double* resid;
  int32_t* status;
};

__global__ void __launch_bounds__(128) k_sip2d(const Sip2dArgs p) {
  const int64_t th = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (th >= p.L.nsys) return;
  const int64_t sys = p.L.sys(th);
  const int64_t nx = p.nx, ny = p.ny, N = nx * ny;
  const int64_t q0 = p.L.base(sys), es = p.L.stride();
  const int64_t w0 = p.W.base(th), ws = p.W.stride();
  auto Q = [&](int64_t k) { return q0 + k * es; };     // input / output element k
  auto Wk = [&](int64_t k) { return w0 + k * ws; };    // scratch element k
  int32_t st = BAND_OK;
  // ---- ILU(0)
  {
    int64_t xk = 0, yk = 0;
    double uc1 = 0.0, e1 = 0.0;      // uc_{k-1}, e_{k-1}
    for (int64_t k = 0; k < N; ++k) {
      double v = ldro(p.c + Q(k));
      double lsk = 0.0, lwk = 0.0;
      if (yk > 0) {
        lsk = ldro(p.s + Q(k)) * p.ruc[Wk(k - nx)];
        v = fma(-lsk, ldro(p.t + Q(k - nx)), v);
      }
      if (xk > 0) {
        lwk = ldro(p.w + Q(k)) * uc1;
        v = fma(-lwk, e1, v);
      }
      if (is_zero(v)) {
        st = BAND_ERR_ZERO_PIVOT;
        break;
      }
      const double r = rcp64(v);
      p.ls[Wk(k)] = lsk;
      p.lw[Wk(k)] = lwk;
      p.ruc[Wk(k)] = r;
      uc1 = r;
      e1 = ldro(p.e + Q(k));
      if (++xk == nx) { xk = 0; ++yk; uc1 = 0.0; e1 = 0.0; }
    }
  }
  int32_t it = 0;
  double rn = 0.0;
  if (st == BAND_OK) {
    for (int64_t k = 0; k < N; ++k) p.x[Q(k)] = 0.0;
    for (;;) {
      // ---- r = f - A x, max |r|
      rn = 0.0;
      {
        int64_t xk = 0, yk = 0;
        double xm = 0.0, x0 = p.x[Q(0)];
        for (int64_t k = 0; k < N; ++k) {
          const double xp = (xk + 1 < nx) ? p.x[Q(k + 1)] : 0.0;
          double ax = ldro(p.c + Q(k)) * x0;
          if (yk > 0) ax = fma(ldro(p.s + Q(k)), p.x[Q(k - nx)], ax);
          if (xk > 0) ax = fma(ldro(p.w + Q(k)), xm, ax);
          if (xk + 1 < nx) ax = fma(ldro(p.e + Q(k)), xp, ax);
          if (yk + 1 < ny) ax = fma(ldro(p.t + Q(k)), p.x[Q(k + nx)], ax);
          const double r = fabs(p.f[Q(k)] - ax);
          if (!(r <= rn)) rn = r;
          xm = x0;
          x0 = xp;
          if (++xk == nx) {
            xk = 0;
            ++yk;
            xm = 0.0;
            x0 = (k + 1 < N) ? p.x[Q(k + 1)] : 0.0;
          }
        }
      }
      if (rn < p.tol || it >= p.max_it || not_finite(rn)) break;
      // ---- forward: L y = K x + f
      {
        int64_t xk = 0, yk = 0;
        double y1 = 0.0;
        for (int64_t k = 0; k < N; ++k) {
          double v = p.f[Q(k)];
          const double lsk = p.ls[Wk(k)], lwk = p.lw[Wk(k)];
          if (yk > 0 && xk + 1 < nx) v = fma(lsk * ldro(p.e + Q(k - nx)), p.x[Q(k - nx + 1)], v);
          if (xk > 0 && yk + 1 < ny) v = fma(lwk * ldro(p.t + Q(k - 1)), p.x[Q(k + nx - 1)], v);
          if (yk > 0) v = fma(-lsk, p.y[Wk(k - nx)], v);
          if (xk > 0) v = fma(-lwk, y1, v);
          p.y[Wk(k)] = v;
          y1 = v;
          if (++xk == nx) { xk = 0; ++yk; y1 = 0.0; }
        }
      }
      // ---- backward: U x = y
      {
        int64_t xk = nx - 1, yk = ny - 1;
        double x1 = 0.0;
        for (int64_t k = N - 1; k >= 0; --k) {
          double v = p.y[Wk(k)];
          if (xk + 1 < nx) v = fma(-ldro(p.e + Q(k)), x1, v);
          if (yk + 1 < ny) v = fma(-ldro(p.t + Q(k)), p.x[Q(k + nx)], v);
          v *= p.ruc[Wk(k)];
          p.x[Q(k)] = v;
          x1 = v;
          if (xk-- == 0) { xk = nx - 1; --yk; x1 = 0.0; }
        }
      }
      ++it;
    }
    if (not_finite(rn)) st = BAND_ERR_NONFINITE;
    else if (!(rn < p.tol)) st = BAND_ERR_NOT_CONVERGED;
  }
  set_status(p.status, sys, st);
  if (p.iters) p.iters[sys] = it;
  if (p.resid) p.resid[sys] = rn;
}

// One warp per system for grids of at most 32 columns: lane x holds column x.  The
// residual pass walks the grid rows (the x +- 1 neighbours by shuffles, the y +- 1 ones
// kept in registers); ILU(0), L y = K x + f and U x = y are recurrences along both grid
// directions ((x, y) needs (x - 1, y) and (x, y - 1), or (x + 1, y) and (x, y + 1)), so
// they run on anti-diagonals x + y = d: at step d lane x takes row y = d - x, its
// neighbour in its own column is its own previous step and its neighbour in its row is
// lane x -+ 1's previous step (one shuffle).  The same arithmetic as k_sip2d, in the
// same order per unknown; a warp's chains are nx + ny - 1 steps instead of nx ny rows,
// and the launch has a warp per system instead of a thread.
__global__ void __launch_bounds__(128) k_sip2d_warp(const Sip2dArgs p) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= p.L.nsys) return;                     // the whole warp
  const unsigned full = 0xffffffffu;
  const int lane = (int)(threadIdx.x & 31);
  const int64_t sys = p.L.sys(t);
  const int nx = (int)p.nx;
  const int64_t ny = p.ny;
  const int64_t q0 = p.L.base(sys), es = p.L.stride();
  auto Q = [&](int64_t k) { return q0 + k * es; };
  // scratch rows laid out like the inputs: interleaved by system (the spill layout:
  // a 32-byte sector then serves four systems, the block's four warps) when the systems
  // are, else each system's nx ny values consecutive (a sector serves one warp's lanes
  // on consecutive wavefronts).  Measured on 16384 grids of 32 x 32: interleaved inputs
  // 19.6 ms against 20.3 with per-system scratch; contiguous 14.2 against 14.4.
  const bool sys_major = p.L.ss != 1;
  const int64_t w0 = sys_major ? t * (int64_t)nx * ny : p.W.base(t);
  const int64_t ws = sys_major ? 1 : p.W.stride();
  auto Wk = [&](int64_t k) { return w0 + k * ws; };
  const bool col = lane < nx;
  const int64_t steps = (int64_t)nx + ny - 1;
  int32_t st = BAND_OK;
  // ---- ILU(0)
  {
    double ruc = 0.0, tt = 0.0, ee = 0.0;      // this lane's last point: 1/uc, t, e
    bool zero = false;
    for (int64_t d = 0; d < steps; ++d) {
      const double ruc_w = __shfl_up_sync(full, ruc, 1), e_w = __shfl_up_sync(full, ee, 1);
      const int64_t y = d - lane;
      if (col && y >= 0 && y < ny && !zero) {
        const int64_t k = y * nx + lane;
        double v = ldro(p.c + Q(k));
        double lsk = 0.0, lwk = 0.0;
        if (y > 0) {
          lsk = ldro(p.s + Q(k)) * ruc;
          v = fma(-lsk, tt, v);
        }
        if (lane > 0) {
          lwk = ldro(p.w + Q(k)) * ruc_w;
          v = fma(-lwk, e_w, v);
        }
        if (is_zero(v)) {
          zero = true;
        } else {
          ruc = rcp64(v);
          p.ls[Wk(k)] = lsk;
          p.lw[Wk(k)] = lwk;
          p.ruc[Wk(k)] = ruc;
          tt = ldro(p.t + Q(k));
          ee = ldro(p.e + Q(k));
        }
      }
    }
    if (__any_sync(full, zero)) st = BAND_ERR_ZERO_PIVOT;
  }
  int32_t it = 0;
  double rn = 0.0;
  if (st == BAND_OK) {
    for (int64_t y = 0; y < ny; ++y)
      if (col) p.x[Q(y * nx + lane)] = 0.0;
    __syncwarp();
    for (;;) {
      // ---- r = f - A x, max |r|
      rn = 0.0;
      {
        double xm = 0.0, x0 = col ? p.x[Q(lane)] : 0.0;
        for (int64_t y = 0; y < ny; ++y) {
          const int64_t k = y * nx + lane;
          const double xp = (col && y + 1 < ny) ? p.x[Q(k + nx)] : 0.0;
          const double xw = __shfl_up_sync(full, x0, 1), xe = __shfl_down_sync(full, x0, 1);
          if (col) {
            double ax = ldro(p.c + Q(k)) * x0;
            if (y > 0) ax = fma(ldro(p.s + Q(k)), xm, ax);
            if (lane > 0) ax = fma(ldro(p.w + Q(k)), xw, ax);
            if (lane + 1 < nx) ax = fma(ldro(p.e + Q(k)), xe, ax);
            if (y + 1 < ny) ax = fma(ldro(p.t + Q(k)), xp, ax);
            rn = max_abs(rn, p.f[Q(k)] - ax);
          }
          xm = x0;
          x0 = xp;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rn = max_abs(rn, __shfl_xor_sync(full, rn, o));
      }
      if (rn < p.tol || it >= p.max_it || not_finite(rn)) break;
      // ---- forward: L y = K x + f (x: the previous iterate, read only here)
      {
        double yy = 0.0, tt = 0.0;               // this lane's last point: y, t
        for (int64_t d = 0; d < steps; ++d) {
          const double y_w = __shfl_up_sync(full, yy, 1), t_w = __shfl_up_sync(full, tt, 1);
          const int64_t y = d - lane;
          if (col && y >= 0 && y < ny) {
            const int64_t k = y * nx + lane;
            double v = p.f[Q(k)];
            const double lsk = p.ls[Wk(k)], lwk = p.lw[Wk(k)];
            if (y > 0 && lane + 1 < nx)
              v = fma(lsk * ldro(p.e + Q(k - nx)), p.x[Q(k - nx + 1)], v);
            if (lane > 0 && y + 1 < ny) v = fma(lwk * t_w, p.x[Q(k + nx - 1)], v);
            if (y > 0) v = fma(-lsk, yy, v);
            if (lane > 0) v = fma(-lwk, y_w, v);
            p.y[Wk(k)] = v;
            yy = v;
            tt = ldro(p.t + Q(k));
          }
        }
      }
      __syncwarp();          // every lane's reads of the previous iterate are done
      // ---- backward: U x = y
      {
        double xx = 0.0;                          // this lane's last point: x
        for (int64_t d = steps - 1; d >= 0; --d) {
          const double x_e = __shfl_down_sync(full, xx, 1);
          const int64_t y = d - lane;
          if (col && y >= 0 && y < ny) {
            const int64_t k = y * nx + lane;
            double v = p.y[Wk(k)];
            if (lane + 1 < nx) v = fma(-ldro(p.e + Q(k)), x_e, v);
            if (y + 1 < ny) v = fma(-ldro(p.t + Q(k)), xx, v);
            v *= p.ruc[Wk(k)];
            p.x[Q(k)] = v;
            xx = v;
          }
        }
      }
      __syncwarp();
      ++it;
    }
    if (not_finite(rn)) st = BAND_ERR_NONFINITE;
    else if (!(rn < p.tol)) st = BAND_ERR_NOT_CONVERGED;
  }
  if (lane == 0) {
    set_status(p.status, sys, st);
    if (p.iters) p.iters[sys] = it;
    if (p.resid) p.resid[sys] = rn;
  }
}

// Copies between the batch's layout and the system-major one (element k of system s at
// s n + k) of up to seven arrays (blockIdx.z): tiles of 32 systems x 32 elements pass
// through shared memory, so the side where consecutive systems are adjacent (the
// interleaved batch) and the side where consecutive elements are (the system-major
// copy) are both read or written along consecutive addresses.
struct Restage {
  const double* src[7];
  double* dst[7];
};
template <bool ToSysMajor>
__global__ void __launch_bounds__(256) k_restage(const __grid_constant__ Restage r, const Layout L) {
  __shared__ double tile[32][33];
  const int64_t n = L.n, nsys = L.nsys, es = L.stride();
  const int64_t s0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const double* src = r.src[blockIdx.z];
  double* dst = r.dst[blockIdx.z];
  const int tx = (int)(threadIdx.x & 31), ty = (int)(threadIdx.x >> 5);
  // tile[j][i]: element k0 + j of system s0 + i
  for (int j = ty; j < 32; j += 8) {
    if (ToSysMajor) {
      const int64_t sy = s0 + tx, k = k0 + j;
      if (sy < nsys && k < n) tile[j][tx] = src[L.base(sy) + k * es];
    } else {
      const int64_t sy = s0 + j, k = k0 + tx;
      if (sy < nsys && k < n) tile[tx][j] = src[sy * n + k];
    }
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    if (ToSysMajor) {
      const int64_t sy = s0 + j, k = k0 + tx;
      if (sy < nsys && k < n) dst[sy * n + k] = tile[tx][j];
    } else {
      const int64_t sy = s0 + tx, k = k0 + j;
      if (sy < nsys && k < n) dst[L.base(sy) + k * es] = tile[j][tx];
    }
  }
}

// Batches whose systems are not stored row-contiguously (elem_stride > 1, e.g.
// interleaved) are staged: the warp kernel's lanes walk a grid row, i.e. consecutive
// elements of one system, and on interleaved data those are nsys elements apart (one
// sector per lane).  The five diagonals, f and x are copied system-major once, the
// kernel runs on the copies (read ~12 times each over the updates), and x is copied
// back.  x goes in too, so that a system whose ILU(0) fails keeps the caller's x.
bool staged(const band_desc* d) { return d->elem_stride != 1 && (d->n + 31) / 32 <= 65535; }

struct Sip2dWs {
  void *ls, *lw, *ruc, *y;
  void* copy[7];      // staged s, w, c, e, t, f, x (system-major), or null
};
Sip2dWs carve_sip2d(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  const size_t rows = (size_t)spill_rows(d) * sizeof(double);
  Sip2dWs w{};
  w.ls = c.take(rows);
  w.lw = c.take(rows);
  w.ruc = c.take(rows);
  w.y = c.take(rows);
  if (staged(d))
    for (int a = 0; a < 7; ++a) w.copy[a] = c.take((size_t)d->nsys * (size_t)d->n * sizeof(double));
  *bytes = c.size();
  return w;
}

}  // namespace

size_t sip2d_workspace_bytes(const band_desc* d) {
  if (d->dtype != BAND_F64 || d->offsets) return 0;
  size_t b = 0;
  carve_sip2d(d, nullptr, &b);
  return b;
}

}  // namespace band

using namespace band;

extern "C" band_status band_sip2d(const band_desc* desc, int64_t nx, const void* const diag[5],
                                  const double* f, double* x, double tol, int32_t max_it,
                                  int32_t* iters, double* resid, int32_t* sys_status, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64 || desc->offsets || desc->hbw) return BAND_ERR_ARG;
  if (desc->schedule != BAND_SCHED_AUTO || desc->chunks) return BAND_ERR_ARG;
  if (nx < 1 || desc->n % nx != 0 || !(tol == tol) || max_it < 0) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !diag[0] || !diag[1] || !diag[2] || !diag[3] || !diag[4] || !f || !x)
    return BAND_ERR_ARG;
  if ((const void*)x == (const void*)f) return BAND_ERR_ARG;
  if (!arrays_aligned(BAND_F64, diag, f, x, sys_status) || !aligned_all(8, {resid}) ||
      !aligned_all(4, {iters}))
    return BAND_ERR_ARG;
  size_t need = 0;
  carve_sip2d(desc, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const Sip2dWs w = carve_sip2d(desc, ws, &need);
  Sip2dArgs p{layout_of(desc), spill_of(desc), nx, desc->n / nx,
              (const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
              (const double*)diag[3], (const double*)diag[4], f, x, (double*)w.ls,
              (double*)w.lw, (double*)w.ruc, (double*)w.y, tol, max_it, iters, resid,
              sys_status};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (nx > 32) {
    k_sip2d<<<(unsigned)((desc->nsys + 127) / 128), 128, 0, st>>>(p);
    return cuda_status(cudaGetLastError());
  }
  if (!staged(desc)) {
    k_sip2d_warp<<<(unsigned)((desc->nsys + 3) / 4), 128, 0, st>>>(p);
    return cuda_status(cudaGetLastError());
  }
  // the system-major copies: s, w, c, e, t, f, x in, the warp kernel, x out
  const Layout L = layout_of(desc);
  const dim3 tiles((unsigned)((desc->nsys + 31) / 32), (unsigned)((desc->n + 31) / 32), 7);
  Restage in{};
  for (int a = 0; a < 5; ++a) in.src[a] = (const double*)diag[a];
  in.src[5] = f;
  in.src[6] = x;
  for (int a = 0; a < 7; ++a) in.dst[a] = (double*)w.copy[a];
  k_restage<true><<<tiles, 256, 0, st>>>(in, L);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  band_desc dm = *desc;
  dm.sys_stride = desc->n;
  dm.elem_stride = 1;
  p.L = layout_of(&dm);
  p.s = in.dst[0]; p.w = in.dst[1]; p.c = in.dst[2]; p.e = in.dst[3]; p.t = in.dst[4];
  p.f = in.dst[5];
  p.x = in.dst[6];
  k_sip2d_warp<<<(unsigned)((desc->nsys + 3) / 4), 128, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  Restage out{};
  out.src[0] = in.dst[6];
  out.dst[0] = x;
  k_restage<false><<<dim3(tiles.x, tiles.y, 1), 256, 0, st>>>(out, L);
  return cuda_status(cudaGetLastError());
}
