// runtime.cu -- host-side batch runtime: size buckets of ragged batches and the
// measuring autotuner of the thread-per-system / two-sided choice.  See include/band.h.
//
// The ADI step solves many independent systems (Veneva & Ayriyan, Sec. 1); ragged
// batches of uneven sizes and mixed bandwidth are cut into buckets so that every
// problem of a band_solve_batch launch has one bandwidth and sizes within a factor of
// two (the warps of a bucket then do similar work, and the two-sided schedule applies).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
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

band_status time_one(const band_problem& q, int32_t schedule, int32_t reps, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1, float* best) {
  band_desc d = *q.desc;
  d.schedule = schedule;
  band_problem p = q;
  p.desc = &d;
  band_status v = band_solve_batch(&p, 1, st);            // warm-up
  if (v != BAND_OK) return v;
  *best = INFINITY;
  for (int r = 0; r < reps; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) return BAND_ERR_CUDA;
    v = band_solve_batch(&p, 1, st);
    if (v != BAND_OK) return v;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
      return BAND_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return BAND_ERR_CUDA;
    *best = std::min(*best, ms);
  }
  return BAND_OK;
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
                                     int32_t* schedules, void* stream) {
  if (count < 0 || count > BAND_MAX_BATCH || (count > 0 && (!probs || !schedules)) || reps < 1)
    return BAND_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!probs[i].desc || !desc_ok(probs[i].desc)) return BAND_ERR_ARG;
  if (count == 0) return BAND_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BAND_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  band_status out = BAND_OK;
  for (int32_t i = 0; i < count && out == BAND_OK; ++i) {
    const band_problem& q = probs[i];
    schedules[i] = q.desc->schedule;
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
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return out;
}

extern "C" void band_autotune_reset(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
}
