// runtime.cu -- host-side batch runtime: size buckets of ragged batches and the
// measuring autotuner of the schedules (thread per system, two-sided, partitioned).
// See include/band.h.
//
// The ADI step solves many independent systems (Veneva & Ayriyan, Sec. 1); ragged
// batches of uneven sizes and mixed bandwidth are cut into buckets so that every
// problem of a band_solve_batch launch has one bandwidth and sizes within a factor of
// two (the warps of a bucket then do similar work, and the two-sided schedule applies).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <sys/stat.h>
#include <tuple>
#include <vector>

#include "api_util.h"
#include "kernels.h"

using namespace band;

namespace {

int log2_floor(int64_t v) {
  int k = 0;
  while (v > 1) {
    v >>= 1;
    ++k;
  }
  return k;
}
int log2_ceil(int64_t v) { return v <= 1 ? 0 : log2_floor(v - 1) + 1; }

// ---------------------------------------------------------------- autotuner cache
using TuneKey = std::tuple<int, int, int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int32_t> g_tune;
bool g_loaded[64];

// The decisions persist in a file of JSON lines, one decision a line, each keyed by the
// GPU (name and compute capability) and the CUDA runtime version:
//   {"gpu": "<name>", "cc": "<major>.<minor>", "cuda": <version>, "kind": "schedule",
//    "key": [dtype, method, half_bw, ceil log2 n, ceil log2 nsys, layout, x is f],
//    "value": <band_schedule>}
//   {"gpu": ..., "kind": "batch_warps", "value": <warps per block of the batched kernel>}
// Later lines override earlier ones.  The file is $BAND_TUNE_CACHE, or
// $HOME/.cache/libband/tune.jsonl when that is unset; an empty BAND_TUNE_CACHE turns
// persistence off.
std::string cache_path() {
  const char* env = std::getenv("BAND_TUNE_CACHE");
  if (env) return std::string(env);
  const char* home = std::getenv("HOME");
  if (!home || !*home) return std::string();
  return std::string(home) + "/.cache/libband/tune.jsonl";
}

struct GpuId {
  std::string name, cc;
  int cuda = 0;
};
bool gpu_id(int dev, GpuId* id) {
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return false;
  id->name = pr.name;
  for (char& ch : id->name)
    if (ch == '"' || ch == '\\') ch = '_';
  id->cc = std::to_string(pr.major) + "." + std::to_string(pr.minor);
  return cudaRuntimeGetVersion(&id->cuda) == cudaSuccess;
}

std::string line_prefix(const GpuId& id) {
  return "{\"gpu\": \"" + id.name + "\", \"cc\": \"" + id.cc + "\", \"cuda\": " +
         std::to_string(id.cuda) + ", ";
}

// Reads this GPU's decisions into the in-process cache (once per device and process).
// Caller holds g_tune_mu.
void load_cache(int dev) {
  if (dev < 0 || dev >= 64 || g_loaded[dev]) return;
  g_loaded[dev] = true;
  const std::string path = cache_path();
  GpuId id;
  if (path.empty() || !gpu_id(dev, &id)) return;
  FILE* fp = std::fopen(path.c_str(), "r");
  if (!fp) return;
  const std::string prefix = line_prefix(id);
  char buf[1024];
  while (std::fgets(buf, sizeof buf, fp)) {
    if (std::strncmp(buf, prefix.c_str(), prefix.size()) != 0) continue;
    const char* rest = buf + prefix.size();
    int k[7], v = 0;
    if (std::sscanf(rest, "\"kind\": \"schedule\", \"key\": [%d, %d, %d, %d, %d, %d, %d], "
                          "\"value\": %d}", &k[0], &k[1], &k[2], &k[3], &k[4], &k[5], &k[6],
                    &v) == 8) {
      if (v >= BAND_SCHED_THREAD && v <= BAND_SCHED_PARTITIONED)
        g_tune[TuneKey{dev, k[0], k[1], k[2], k[3], k[4], k[5], k[6]}] = v;
    } else if (std::sscanf(rest, "\"kind\": \"batch_warps\", \"value\": %d}", &v) == 1) {
      set_batch_warps(dev, v);
    }
  }
  std::fclose(fp);
}

void mkdirs_for(const std::string& path) {
  for (size_t i = 1; i < path.size(); ++i)
    if (path[i] == '/') mkdir(path.substr(0, i).c_str(), 0755);
}

// Appends lines of decisions for this GPU (best effort: a file that cannot be written
// leaves the in-process cache as the only one).
void save_lines(int dev, const std::vector<std::string>& bodies) {
  const std::string path = cache_path();
  GpuId id;
  if (bodies.empty() || path.empty() || !gpu_id(dev, &id)) return;
  mkdirs_for(path);
  FILE* fp = std::fopen(path.c_str(), "a");
  if (!fp) return;
  const std::string prefix = line_prefix(id);
  for (const std::string& b : bodies) std::fprintf(fp, "%s%s}\n", prefix.c_str(), b.c_str());
  std::fclose(fp);
}

std::string schedule_line(const TuneKey& k, int32_t v) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "\"kind\": \"schedule\", \"key\": [%d, %d, %d, %d, %d, %d, %d], "
                                 "\"value\": %d",
                std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                std::get<6>(k), std::get<7>(k), (int)v);
  return buf;
}

int layout_class(const band_desc* d) {
  if (d->offsets) return 0;                    // ragged (packed rows, one system a lane)
  if (d->sys_stride == 1) return 1;            // interleaved
  if (d->elem_stride == 1) return 2;           // contiguous
  return 3;                                    // general strides
}

TuneKey tune_key(int dev, const band_problem& q) {
  const band_desc* d = q.desc;
  return TuneKey{dev, d->dtype, q.method, d->half_bw, log2_ceil(d->n), log2_ceil(d->nsys),
                 layout_class(d), q.x == q.f ? 1 : 0};
}

// A problem the tuner may decide: a fused direct solve of one bandwidth on AUTO.
bool tunable(const band_problem& q) {
  if (q.op != BAND_OP_SOLVE || !q.desc || q.desc->nsys == 0) return false;
  if (q.desc->schedule != BAND_SCHED_AUTO || q.desc->hbw) return false;
  return kmode_for(q.desc, q.method) > 0;
}

// Best of `reps` timed band_solve_batch launches of the list, after one warm-up.
band_status time_batch(const band_problem* p, int32_t count, int32_t reps, cudaStream_t st,
                       cudaEvent_t e0, cudaEvent_t e1, float* best) {
  band_status v = band_solve_batch(p, count, st);            // warm-up
  if (v != BAND_OK) return v;
  *best = INFINITY;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return BAND_ERR_CUDA;
    v = band_solve_batch(p, count, st);
    if (v != BAND_OK) return v;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return BAND_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return BAND_ERR_CUDA;
    *best = std::min(*best, ms);
  }
  return BAND_OK;
}

band_status time_one(const band_problem& q, int32_t schedule, int32_t reps, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1, float* best) {
  band_desc d = *q.desc;
  d.schedule = schedule;
  band_problem p = q;
  p.desc = &d;
  return time_batch(&p, 1, reps, st, e0, e1, best);
}

// A move of the joint phase has to gain this fraction of the launch time to be kept.
constexpr float kJointGain = 0.02f;
// Passes of the joint search over the partitioned moves.
constexpr int kJointPasses = 4;

// Row diagonal dominance, |c_i| >= |a_i| + |b_i| + |d_i| + |e_i| (the entries inside the
// matrix) for every row of every system, one thread per system; a row that fails
// (NaN included) sets *bad.
template <typename T, int K>
__global__ void __launch_bounds__(128) k_dominance(const Layout L, const T* a, const T* b,
                                                   const T* c, const T* d, const T* e, int* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L.nsys) return;
  const int64_t s = L.sys(t);
  const int64_t n = L.rows(s), q0 = L.base(s), es = L.stride();
  bool ok = true;
  for (int64_t i = 0; i < n && ok; ++i) {
    const int64_t q = q0 + i * es;
    T off = (i >= 1 ? fabs(b[q]) : T(0)) + (i + 1 < n ? fabs(d[q]) : T(0));
    if (K == 2) off += (i >= 2 ? fabs(a[q]) : T(0)) + (i + 2 < n ? fabs(e[q]) : T(0));
    ok = fabs(c[q]) >= off;
  }
  if (!ok) atomicOr(bad, 1);
}

// Is every system of the problem row diagonally dominant?  (-1: CUDA error)  The flag
// lives in the first bytes of the problem's own workspace, which holds nothing between
// calls.
int dominant(const band_problem& q, cudaStream_t st) {
  int* flag = static_cast<int*>(q.ws);
  const band_desc* d = q.desc;
  const Layout L = layout_of(d);
  const int K = kmode_for(d, q.method);
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return -1;
  const unsigned grid = (unsigned)((d->nsys + 127) / 128);
  if (d->dtype == BAND_F64) {
    const double* g[5];
    for (int j = 0; j < 5; ++j) g[j] = static_cast<const double*>(q.diag[j]);
    if (K == 2) k_dominance<double, 2><<<grid, 128, 0, st>>>(L, g[0], g[1], g[2], g[3], g[4], flag);
    else k_dominance<double, 1><<<grid, 128, 0, st>>>(L, g[0], g[1], g[2], g[3], g[4], flag);
  } else {
    const float* g[5];
    for (int j = 0; j < 5; ++j) g[j] = static_cast<const float*>(q.diag[j]);
    if (K == 2) k_dominance<float, 2><<<grid, 128, 0, st>>>(L, g[0], g[1], g[2], g[3], g[4], flag);
    else k_dominance<float, 1><<<grid, 128, 0, st>>>(L, g[0], g[1], g[2], g[3], g[4], flag);
  }
  int h = 1;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return -1;
  return h == 0 ? 1 : 0;
}

}  // namespace

extern "C" int32_t band_plan_ragged(const int64_t* offsets, const int8_t* hbw, int32_t half_bw,
                                    int64_t nsys, int64_t* order, band_bucket* buckets,
                                    int32_t max_buckets) {
  if (nsys < 0 || !offsets || (nsys > 0 && !order) || max_buckets < 0) return -1;
  if (!hbw && half_bw != 1 && half_bw != 2) return -1;
  if (nsys == 0) return 0;
  struct Key {
    int8_t k;
    int8_t lg;
    int64_t n;
    int64_t id;
  };
  std::vector<Key> keys((size_t)nsys);
  for (int64_t s = 0; s < nsys; ++s) {
    const int64_t n = offsets[s + 1] - offsets[s];
    const int k = hbw ? hbw[s] : half_bw;
    if (n < 1 || (k != 1 && k != 2)) return -1;
    keys[(size_t)s] = Key{(int8_t)k, (int8_t)log2_floor(n), n, s};
  }
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.k != b.k) return a.k < b.k;
    if (a.lg != b.lg) return a.lg > b.lg;        // larger buckets first
    if (a.n != b.n) return a.n > b.n;            // within a bucket, longest first
    return a.id < b.id;
  });
  int32_t nb = 0;
  for (int64_t i = 0; i < nsys; ++i) {
    const Key& key = keys[(size_t)i];
    order[i] = key.id;
    const bool fresh = i == 0 || key.k != keys[(size_t)i - 1].k || key.lg != keys[(size_t)i - 1].lg;
    if (fresh) {
      if (nb >= max_buckets) return -1;
      if (buckets) buckets[nb] = band_bucket{i, 0, key.n, key.k, 0};
      ++nb;
    }
    if (buckets) ++buckets[nb - 1].count;
  }
  return nb;
}

extern "C" band_status band_autotune(const band_problem* probs, int32_t count, int32_t reps,
                                     int32_t flags, int32_t* schedules, int32_t* chunks,
                                     void* stream) {
  if (count < 0 || count > BAND_MAX_BATCH || (count > 0 && (!probs || !schedules)) || reps < 1)
    return BAND_ERR_ARG;
  if (flags & ~BAND_TUNE_JOINT) return BAND_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!probs[i].desc || !desc_ok(probs[i].desc)) return BAND_ERR_ARG;
  if (count == 0) return BAND_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BAND_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  band_status out = BAND_OK;
  for (int32_t i = 0; i < count; ++i) {
    schedules[i] = probs[i].desc->schedule;
    if (chunks) chunks[i] = probs[i].desc->chunks;
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache(dev);
  }
  std::vector<std::string> fresh;      // decisions to persist
  // per problem: thread per system or two-sided, timed alone (cached)
  for (int32_t i = 0; i < count && out == BAND_OK; ++i) {
    const band_problem& q = probs[i];
    if (!tunable(q)) continue;
    const TuneKey key = tune_key(dev, q);
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      const auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        schedules[i] = it->second;
        continue;
      }
    }
    if (!e0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
      out = BAND_ERR_CUDA;
      break;
    }
    float t_thread = 0.f, t_two = 0.f;
    out = time_one(q, BAND_SCHED_THREAD, reps, st, e0, e1, &t_thread);
    if (out != BAND_OK) break;
    out = time_one(q, BAND_SCHED_TWO_SIDED, reps, st, e0, e1, &t_two);
    if (out != BAND_OK) break;
    const int32_t pick = t_two < t_thread ? BAND_SCHED_TWO_SIDED : BAND_SCHED_THREAD;
    schedules[i] = pick;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = pick;
    fresh.push_back(schedule_line(key, pick));
  }
  // joint: the whole list as one launch; problems move to the partitioned schedule,
  // longest systems first, while that shortens the launch
  if (out == BAND_OK && (flags & BAND_TUNE_JOINT)) {
    std::vector<band_desc> descs((size_t)count);
    std::vector<band_problem> list(probs, probs + count);
    std::vector<int32_t> cand;
    for (int32_t i = 0; i < count && out == BAND_OK; ++i) {
      descs[(size_t)i] = *probs[i].desc;
      list[(size_t)i].desc = &descs[(size_t)i];
      if (!tunable(probs[i])) continue;
      descs[(size_t)i].schedule = schedules[i];
      band_desc dp = *probs[i].desc;
      dp.schedule = BAND_SCHED_PARTITIONED;
      dp.chunks = 0;
      size_t need = 0;
      carve_solve(&dp, probs[i].method, nullptr, &need);
      if (need > probs[i].ws_bytes || dp.n < 64 || !probs[i].ws) continue;
      const int dom = dominant(probs[i], st);
      if (dom < 0) out = BAND_ERR_CUDA;
      else if (dom) cand.push_back(i);
    }
    std::stable_sort(cand.begin(), cand.end(),
                     [&](int32_t x, int32_t y) { return probs[x].desc->n > probs[y].desc->n; });
    if (!cand.empty() && !e0 &&
        (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
      out = BAND_ERR_CUDA;
    float base = 0.f;
    if (out == BAND_OK && !cand.empty())
      out = time_batch(list.data(), count, reps, st, e0, e1, &base);
    // passes over the candidates not yet moved, until a pass moves none: a move that
    // gains nothing while a longer chain elsewhere bounds the launch can gain once that
    // chain is cut (a ragged bucket of one 8192-row system after the 8190-row bucket)
    std::vector<char> moved(cand.size(), 0);
    for (int pass = 0; pass < kJointPasses && out == BAND_OK; ++pass) {
      int misses = 0, moves = 0;
      for (size_t c = 0; c < cand.size() && out == BAND_OK && misses < 2; ++c) {
        if (moved[c]) continue;
        band_desc& d = descs[(size_t)cand[c]];
        const band_desc keep = d;
        int best_p = 0;
        float best_t = base * (1.f - kJointGain);
        for (int P = 8; P <= 32 && out == BAND_OK; P *= 2) {
          if (d.n < (int64_t)16 * P) break;
          d.schedule = BAND_SCHED_PARTITIONED;
          d.chunks = P;
          float tm = 0.f;
          out = time_batch(list.data(), count, reps, st, e0, e1, &tm);
          if (tm < best_t) { best_t = tm; best_p = P; }
        }
        d = keep;
        if (out != BAND_OK) break;
        if (best_p) {
          d.schedule = BAND_SCHED_PARTITIONED;
          d.chunks = best_p;
          base = best_t;
          moved[c] = 1;
          misses = 0;
          ++moves;
        } else {
          ++misses;
        }
      }
      if (moves == 0) break;
    }
    for (int32_t i = 0; i < count && out == BAND_OK; ++i) {
      schedules[i] = descs[(size_t)i].schedule;
      if (chunks) chunks[i] = descs[(size_t)i].chunks;
    }
    // the block size of the batched kernel: the whole list at 1, 2 and 4 warps per
    // block, with the schedules just chosen (kept per device)
    if (out == BAND_OK) {
      if (!e0 && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        out = BAND_ERR_CUDA;
      const int keep_w = batch_warps(dev);
      int best_w = keep_w;
      float best_t = INFINITY;
      for (int w = 1; w <= 4 && out == BAND_OK; w *= 2) {
        set_batch_warps(dev, w);
        float tm = 0.f;
        out = time_batch(list.data(), count, reps, st, e0, e1, &tm);
        if (tm < best_t) { best_t = tm; best_w = w; }
      }
      set_batch_warps(dev, out == BAND_OK ? best_w : keep_w);
      if (out == BAND_OK) fresh.push_back("\"kind\": \"batch_warps\", \"value\": " +
                                         std::to_string(best_w));
    }
  }
  if (out == BAND_OK) save_lines(dev, fresh);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return out;
}

extern "C" int32_t band_batch_warps(int32_t device) {
  return (device >= 0 && device < 64) ? batch_warps(device) : -1;
}

extern "C" void band_autotune_reset(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  for (int d = 0; d < 64; ++d) {
    g_loaded[d] = false;
    set_batch_warps(d, 2);
  }
}
