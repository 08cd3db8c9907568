// direct.cu -- NTDM / NPDM (LU without pivoting) and STDM / SPDM (symbolic zero
// pivots) for batches of independent band systems, one thread per system.
//
// Veneva & Ayriyan, arXiv:1804.09666: the direct numerical methods NPDM/NTDM and
// the symbolic methods SPDM/STDM (Sec. 1; costs in Table 7).  The PD recurrence,
// with U unit upper and every quantity with a negative index zero:
//   gamma_i = b_i - alpha_{i-2} a_i
//   mu_i    = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i
//   alpha_i = (d_i - beta_{i-1} gamma_i) / mu_i,   beta_i = e_i / mu_i
//   z_i     = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i
//   x_i     = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
// (TD: a = e = 0).  Each mu_i is inverted once and used by multiplication.  The
// forward sweep keeps alpha, beta in the workspace (interleaved by system) and z in
// x (numeric methods) or in the workspace too (symbolic methods, so that a system
// handed to the fix-up pass still has an intact f when x aliases f); the backward
// sweep writes x.
#include "common.cuh"
#include "kernels.h"
#include "partition.cuh"
#include "sweeps.cuh"
#include "symbolic.cuh"

namespace band {

// positions a thread / two-sided launch covers (DirectArgs::nsys_dev)
template <typename T>
__device__ __forceinline__ bool in_batch(const DirectArgs<T>& p, int64_t t) {
  return t < p.L.nsys && (!p.nsys_dev || (unsigned long long)t < *p.nsys_dev);
}

// ---------------------------------------------------------------------------
// fused factor + solve (device function in sweeps.cuh)
// ---------------------------------------------------------------------------
template <typename T, int K>
__global__ void __launch_bounds__(32 * SweepWarps<T>::value, kSweepWarpsPerSm / SweepWarps<T>::value)
    k_direct(const DirectArgs<T> p) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (!in_batch(p, t)) return;
  void* stage = stage_mem + (threadIdx.x >> 5) * stage_bytes_per_warp<T>();
  if (K == 0) {
    if (p.L.kband(p.L.sys(t)) == 1) direct_one<T, 1>(p, t, stage);
    else direct_one<T, 2>(p, t, stage);
  } else {
    direct_one<T, K>(p, t, stage);
  }
}

template <typename T>
cudaError_t launch_direct(const DirectArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 32 * SweepWarps<T>::value;
  const size_t smem = (size_t)SweepWarps<T>::value * stage_bytes_per_warp<T>();
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_direct<T, 1><<<grid, tb, smem, st>>>(p);
  else if (kmode == 2) k_direct<T, 2><<<grid, tb, smem, st>>>(p);
  else k_direct<T, 0><<<grid, tb, smem, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_direct<double>(const DirectArgs<double>&, int, cudaStream_t);
template cudaError_t launch_direct<float>(const DirectArgs<float>&, int, cudaStream_t);

// two threads (lanes l, l ^ 16) per system; one bandwidth for the batch
template <typename T, int K>
__global__ void __launch_bounds__(32 * SweepWarps<T>::value, kSweepWarpsPerSm / SweepWarps<T>::value)
    k_twisted(const DirectArgs<T> p) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  void* stage = stage_mem + (threadIdx.x >> 5) * stage_bytes_per_warp<T>();
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t t = warp * 16 + (threadIdx.x & 15);
  twisted_one<T, K>(p, t, in_batch(p, t), stage);
}

template <typename T>
cudaError_t launch_twisted(const DirectArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int64_t threads = (p.L.nsys + 15) / 16 * 32;
  const int tb = 32 * SweepWarps<T>::value;
  const unsigned grid = (unsigned)((threads + tb - 1) / tb);
  const size_t smem = (size_t)SweepWarps<T>::value * stage_bytes_per_warp<T>();
  if (kmode == 1) k_twisted<T, 1><<<grid, tb, smem, st>>>(p);
  else if (kmode == 2) k_twisted<T, 2><<<grid, tb, smem, st>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}
template cudaError_t launch_twisted<double>(const DirectArgs<double>&, int, cudaStream_t);
template cudaError_t launch_twisted<float>(const DirectArgs<float>&, int, cudaStream_t);

// P lanes per system, 32 / P systems per warp (partition.cuh); one bandwidth
template <typename T, int K, int P>
__global__ void __launch_bounds__(32 * SweepWarps<T>::value) k_partition(const DirectArgs<T> p) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  T* stage = reinterpret_cast<T*>(stage_mem + (threadIdx.x >> 5) * stage_bytes_per_warp<T>());
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  partition_one<T, K, P>(p, warp, stage);
}

// one system per block of W warps (P = 32 W chunks)
template <typename T, int K, int W>
__global__ void __launch_bounds__(32 * W) k_partition_block(const DirectArgs<T> p) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  partition_block<T, K, W>(p, stage_mem);
}

template <typename T, int K>
static cudaError_t launch_partition_k(const DirectArgs<T>& p, int parts, unsigned grid, int tb,
                                      size_t smem, cudaStream_t st) {
  switch (parts) {
    case 4: k_partition<T, K, 4><<<grid, tb, smem, st>>>(p); break;
    case 8: k_partition<T, K, 8><<<grid, tb, smem, st>>>(p); break;
    case 16: k_partition<T, K, 16><<<grid, tb, smem, st>>>(p); break;
    case 32: k_partition<T, K, 32><<<grid, tb, smem, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int K>
static cudaError_t launch_partition_block_k(const DirectArgs<T>& p, int parts, cudaStream_t st) {
  const unsigned grid = (unsigned)p.L.nsys;
  const size_t smem = (size_t)(parts / 32) * stage_bytes_per_warp<T>();
  switch (parts) {
    case 64: k_partition_block<T, K, 2><<<grid, 64, smem, st>>>(p); break;
    case 128: k_partition_block<T, K, 4><<<grid, 128, smem, st>>>(p); break;
    case 256: {     // 48 KiB of staging areas: the most a launch gets without opting in
      const cudaError_t e = tail_prepare((const void*)k_partition_block<T, K, 8>);
      if (e != cudaSuccess) return e;
      k_partition_block<T, K, 8><<<grid, 256, smem, st>>>(p);
      break;
    }
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_partition(const DirectArgs<T>& p, int kmode, int parts, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  if (parts == 64 || parts == 128 || parts == 256) {
    if (kmode == 1) return launch_partition_block_k<T, 1>(p, parts, st);
    if (kmode == 2) return launch_partition_block_k<T, 2>(p, parts, st);
    return cudaErrorInvalidValue;
  }
  if (parts != 4 && parts != 8 && parts != 16 && parts != 32) return cudaErrorInvalidValue;
  const int64_t warps = (p.L.nsys + 32 / parts - 1) / (32 / parts);
  const int wpb = SweepWarps<T>::value;
  const unsigned grid = (unsigned)((warps + wpb - 1) / wpb);
  const size_t smem = (size_t)wpb * stage_bytes_per_warp<T>();
  if (kmode == 1) return launch_partition_k<T, 1>(p, parts, grid, 32 * wpb, smem, st);
  if (kmode == 2) return launch_partition_k<T, 2>(p, parts, grid, 32 * wpb, smem, st);
  return cudaErrorInvalidValue;
}
template cudaError_t launch_partition<double>(const DirectArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_partition<float>(const DirectArgs<float>&, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// factorisation only: gamma, 1/mu, alpha, beta per row (interleaved like the spill)
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void factor_one(const FactorArgs<T>& p, int64_t s) {
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), wst = p.W.stride();
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T bi = ldro(p.b + q);
    const T ci = ldro(p.c + q);
    T di = ldro(p.d + q);
    bi = (i >= 1) ? bi : T(0);
    di = (i + 1 < n) ? di : T(0);
    T ai = 0, ei = 0;
    if (K == 2) {
      ai = ldro(p.a + q);
      ei = ldro(p.e + q);
      ai = (i >= 2) ? ai : T(0);
      ei = (i + 2 < n) ? ei : T(0);
    }
    const T g = fma(-al2, ai, bi);
    const T m = fma(-al1, g, fma(-be2, ai, ci));
    if (m == T(0)) {
      set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
      return;
    }
    const T r = rcp<T>(m);
    const T alv = fma(-be1, g, di) * r;
    const T bev = ei * r;
    p.gam[w] = g;
    p.rmu[w] = r;
    p.al[w] = alv;
    p.be[w] = bev;
    al2 = al1; al1 = alv; be2 = be1; be1 = bev;
  }
  set_status(p.status, s, BAND_OK);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) k_factor(const FactorArgs<T> p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (K == 0) {
    if (p.L.kband(s) == 1) factor_one<T, 1>(p, s);
    else factor_one<T, 2>(p, s);
  } else {
    factor_one<T, K>(p, s);
  }
}

template <typename T>
cudaError_t launch_factor(const FactorArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 128;
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_factor<T, 1><<<grid, tb, 0, st>>>(p);
  else if (kmode == 2) k_factor<T, 2><<<grid, tb, 0, st>>>(p);
  else k_factor<T, 0><<<grid, tb, 0, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_factor<double>(const FactorArgs<double>&, int, cudaStream_t);
template cudaError_t launch_factor<float>(const FactorArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// solve with stored factors: z_i = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i,
// x_i = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void fsolve_one(const FactoredArgs<T>& p, int64_t s) {
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), wst = p.W.stride();
  T z1 = 0, z2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T zz = p.f[q];
    if (K == 2) {
      T ai = ldro(p.a + q);
      ai = (i >= 2) ? ai : T(0);
      zz = fma(-z2, ai, zz);
    }
    const T zv = fma(-z1, ldro(p.gam + w), zz) * ldro(p.rmu + w);
    p.x[q] = zv;
    z2 = z1;
    z1 = zv;
  }
  T x1 = 0, x2 = 0;
  bool bad = false;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T xi = fma(-ldro(p.al + w), x1, p.x[q]);
    if (K == 2) xi = fma(-ldro(p.be + w), x2, xi);
    p.x[q] = xi;
    bad |= !finite(xi);
    x2 = x1;
    x1 = xi;
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) k_fsolve(const FactoredArgs<T> p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (K == 0) {
    if (p.L.kband(s) == 1) fsolve_one<T, 1>(p, s);
    else fsolve_one<T, 2>(p, s);
  } else {
    fsolve_one<T, K>(p, s);
  }
}

template <typename T>
cudaError_t launch_fsolve(const FactoredArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 128;
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_fsolve<T, 1><<<grid, tb, 0, st>>>(p);
  else if (kmode == 2) k_fsolve<T, 2><<<grid, tb, 0, st>>>(p);
  else k_fsolve<T, 0><<<grid, tb, 0, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_fsolve<double>(const FactoredArgs<double>&, int, cudaStream_t);
template cudaError_t launch_fsolve<float>(const FactoredArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// STDM / SPDM fix-up of the systems whose numeric sweep met an exact zero pivot:
// Laurent series in one symbol t, one warp per system (symbolic.cuh).  Warp w of the
// launch takes the flagged systems w, w + nslots, ... of the list; each warp owns one
// slot of series rows in the workspace.
// ---------------------------------------------------------------------------
constexpr int kFixWarps = 4;

__global__ void __launch_bounds__(32 * kFixWarps) k_symbolic_fixup(const SymArgs p) {
  __shared__ lser::dd stage[kFixWarps][128];
  const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slot >= p.nslots) return;
  const unsigned long long count = *p.fix_count;
  const lser::SlotView sv = lser::slot_view(p, slot);
  for (unsigned long long item = slot; item < count; item += p.nslots)
    lser::symbolic_warp(p, p.fix_list[item], sv, stage[threadIdx.x >> 5]);
}

cudaError_t launch_symbolic_fixup(const SymArgs& p, cudaStream_t st) {
  if (p.nslots <= 0) return cudaSuccess;
  const int64_t threads = p.nslots * 32;
  const int tb = 32 * kFixWarps;
  k_symbolic_fixup<<<(unsigned)((threads + tb - 1) / tb), tb, 0, st>>>(p);
  return cudaGetLastError();
}

size_t symbolic_slot_bytes(int64_t nmax) { return lser::slot_bytes(nmax); }

}  // namespace band
