// atlas_rt_host.cu -- continuous ingest (a cyclic buffer of int16 samples in
// device memory) and the high-level scheduler of Section 2.2 (searching and
// tracking tasks, half of the work each in an amortised sense), built on the
// FSK search's C ABI.  Host code only: a searching task is a search run
// (atlas_fsk_run_codes) on one block copied out of the cyclic buffer; a
// tracking task is one launch of a captured graph that reads its block from the
// cyclic buffer directly (atlas_fsk_tracker_run).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "atlas_fsk.h"
#include "atlas_rt.h"

struct atlas_rt {
  atlas_fsk_t fsk = nullptr;
  int C = 0;
  atlas_rt_opts o = {};
  std::vector<double> period;
  std::vector<int> n_c;    // support of d_c per code
  // cyclic buffer: absolute sample i lives at i % cap
  int16_t* d_ring = nullptr;
  int64_t cap = 0;
  int64_t head = 0;        // absolute index of the next sample to arrive
  int16_t* d_stage = nullptr;  // one task block, contiguous
  atlas_fsk_detection* d_out = nullptr;
  int* d_count = nullptr;
  atlas_fsk_detection* h_out = nullptr;  // pinned
  int* h_count = nullptr;                // pinned
  // scheduler state
  int64_t search_pos = 0;  // absolute start of the next searching block
  std::vector<int> tracking;     // 1: the code is in the tracking queue
  std::vector<double> pred;      // predicted arrival of its next transmission (absolute samples)
  std::vector<int> misses;
  atlas_rt_stats st = {};
  // one single-launch tracker (captured graph) per support length, made on first use
  std::map<int, atlas_fsk_tracker_t> trackers;
  std::string last_error;
};

namespace {

constexpr int kEagerRecords = 8;  // records read back with the count

int fail_cuda(atlas_rt* rt, cudaError_t e) {
  if (rt) rt->last_error = cudaGetErrorString(e);
  return ATLAS_ERR_CUDA;
}

#define CK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return fail_cuda(rt, e_); \
  } while (0)

void free_rt(atlas_rt* rt) {
  if (!rt) return;
  for (auto& kv : rt->trackers) atlas_fsk_tracker_destroy(kv.second);
  cudaFree(rt->d_ring);
  cudaFree(rt->d_stage);
  cudaFree(rt->d_out);
  cudaFree(rt->d_count);
  cudaFreeHost(rt->h_out);
  cudaFreeHost(rt->h_count);
  delete rt;
}

// Copy the block [s, s + len) of absolute samples out of the cyclic buffer.
int stage_block(atlas_rt* rt, cudaStream_t st, int64_t s, int64_t len) {
  const int64_t pos = s % rt->cap;
  const int64_t first = std::min(len, rt->cap - pos);
  CK(cudaMemcpyAsync(rt->d_stage, rt->d_ring + 2 * pos, sizeof(int16_t) * 2 * (size_t)first,
                     cudaMemcpyDeviceToDevice, st));
  if (first < len)
    CK(cudaMemcpyAsync(rt->d_stage + 2 * first, rt->d_ring, sizeof(int16_t) * 2 * (size_t)(len - first),
                       cudaMemcpyDeviceToDevice, st));
  return ATLAS_OK;
}

// One search run on a staged block; leaves the records in h_out, returns the count.
int run_block(atlas_rt* rt, cudaStream_t st, int64_t s, int64_t len, const std::vector<int>& codes, int* n_det) {
  int r = stage_block(rt, st, s, len);
  if (r != ATLAS_OK) return r;
  r = atlas_fsk_run_codes(rt->fsk, st, rt->d_stage, len, s, codes.data(), (int32_t)codes.size(), rt->d_out,
                          rt->o.capacity, rt->d_count);
  if (r != ATLAS_OK) {
    rt->last_error = atlas_fsk_last_error(rt->fsk);
    return r;
  }
  // the count and the first few records come back together (one synchronisation
  // for a tracking task); more records, if there are more, after it
  const int first = std::min(kEagerRecords, rt->o.capacity);
  CK(cudaMemcpyAsync(rt->h_count, rt->d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rt->h_out, rt->d_out, sizeof(atlas_fsk_detection) * (size_t)first, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int n = std::min(*rt->h_count, rt->o.capacity);
  if (n > first) {
    CK(cudaMemcpyAsync(rt->h_out + first, rt->d_out + first, sizeof(atlas_fsk_detection) * (size_t)(n - first),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  *n_det = n;
  return ATLAS_OK;
}

// A tracking task: one graph launch that reads its block straight from the
// cyclic buffer; the records land in h_out.
int run_track(atlas_rt* rt, cudaStream_t st, int c, int64_t s, int* n_det) {
  atlas_fsk_tracker_t& t = rt->trackers[rt->n_c[c]];
  if (!t) {
    const int r = atlas_fsk_tracker_create(&t, rt->fsk, c, rt->o.track_block, rt->d_ring, rt->cap);
    if (r != ATLAS_OK) {
      rt->last_error = atlas_fsk_last_error(rt->fsk);
      t = nullptr;
      return r;
    }
  }
  int32_t n = 0;
  const int r = atlas_fsk_tracker_run(t, st, c, s, rt->h_out, rt->o.capacity, &n);
  if (r != ATLAS_OK) {
    rt->last_error = atlas_fsk_last_error(rt->fsk);
    return r;
  }
  *n_det = std::min<int>(n, rt->o.capacity);
  return ATLAS_OK;
}

struct EventSink {
  atlas_rt_event* ev;
  int cap;
  int n = 0;
  void add(const atlas_rt_event& e) {
    if (n < cap) ev[n] = e;
    ++n;
  }
};

atlas_rt_event make_event(int kind, int code, int64_t start, double toa, int misses) {
  atlas_rt_event e;
  memset(&e, 0, sizeof(e));
  e.kind = kind;
  e.code = code;
  e.task_start = start;
  e.toa = toa;
  e.misses = misses;
  return e;
}

// Tracking block of code c: track_block samples centred on the prediction's support.
int64_t track_start(const atlas_rt* rt, int c) {
  const int64_t margin = (rt->o.track_block - rt->n_c[c]) / 2;
  return std::max<int64_t>(0, llround(rt->pred[c]) - margin);
}

void miss(atlas_rt* rt, int c) {
  rt->pred[c] += rt->period[c];
  if (++rt->misses[c] >= rt->o.max_misses) rt->tracking[c] = 0;  // back to the searching queue
}

}  // namespace

extern "C" {

void atlas_rt_default_opts(atlas_rt_opts* o, double fs_hz) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->ring_samples = (int64_t)llround(16.0 * fs_hz);
  o->search_block = (int32_t)llround(0.1 * fs_hz);
  o->search_overlap = (int32_t)llround(0.01 * fs_hz);
  o->track_block = (int32_t)llround(0.012 * fs_hz);
  o->max_misses = 3;
  o->capacity = 1024;
}

int atlas_rt_create(atlas_rt_t* out, atlas_fsk_t fsk, const double* period_samples, int32_t n_codes,
                    const atlas_rt_opts* opts) {
  if (!out) return ATLAS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!fsk || !period_samples || n_codes <= 0 || !opts) return ATLAS_ERR_INVALID_ARG;
  const atlas_rt_opts& o = *opts;
  std::vector<int> nc(n_codes);
  int max_nc = 0;
  for (int c = 0; c < n_codes; ++c) {
    if (!(period_samples[c] > 0.0) || !isfinite(period_samples[c])) return ATLAS_ERR_INVALID_ARG;
    int32_t W, hop, N, sup;
    if (atlas_fsk_windows(fsk, c, 1, &W, &hop, &N, &sup) != ATLAS_OK) return ATLAS_ERR_INVALID_ARG;
    nc[c] = sup;
    max_nc = std::max(max_nc, sup);
  }
  if (o.search_overlap < max_nc || o.search_block <= o.search_overlap || o.track_block < max_nc ||
      o.ring_samples < (int64_t)o.search_block + o.track_block || o.max_misses < 1 || o.capacity < 1)
    return ATLAS_ERR_INVALID_ARG;
  atlas_rt* rt = new (std::nothrow) atlas_rt();
  if (!rt) return ATLAS_ERR_NO_MEMORY;
  rt->fsk = fsk;
  rt->C = n_codes;
  rt->o = o;
  rt->period.assign(period_samples, period_samples + n_codes);
  rt->n_c = nc;
  rt->cap = o.ring_samples;
  rt->tracking.assign(n_codes, 0);
  rt->pred.assign(n_codes, 0.0);
  rt->misses.assign(n_codes, 0);
  const int64_t stage = std::max<int64_t>(o.search_block, o.track_block);
  if (cudaMalloc((void**)&rt->d_ring, sizeof(int16_t) * 2 * (size_t)rt->cap) != cudaSuccess ||
      cudaMalloc((void**)&rt->d_stage, sizeof(int16_t) * 2 * (size_t)stage) != cudaSuccess ||
      cudaMalloc((void**)&rt->d_out, sizeof(atlas_fsk_detection) * (size_t)o.capacity) != cudaSuccess ||
      cudaMalloc((void**)&rt->d_count, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&rt->h_out, sizeof(atlas_fsk_detection) * (size_t)o.capacity) != cudaSuccess ||
      cudaMallocHost((void**)&rt->h_count, sizeof(int)) != cudaSuccess) {
    free_rt(rt);
    return ATLAS_ERR_NO_MEMORY;
  }
  *out = rt;
  return ATLAS_OK;
}

int atlas_rt_push(atlas_rt_t rt, void* stream, const int16_t* h_iq, int64_t n) {
  if (!rt || n < 0 || (n > 0 && !h_iq)) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t skip = 0;
  if (n > rt->cap) {  // only the newest cap samples survive
    skip = n - rt->cap;
    rt->head += skip;
  }
  int64_t done = skip;
  while (done < n) {
    const int64_t pos = rt->head % rt->cap;
    const int64_t m = std::min(n - done, rt->cap - pos);
    CK(cudaMemcpyAsync(rt->d_ring + 2 * pos, h_iq + 2 * done, sizeof(int16_t) * 2 * (size_t)m,
                       cudaMemcpyHostToDevice, st));
    rt->head += m;
    done += m;
  }
  CK(cudaStreamSynchronize(st));  // the caller's buffer has been read
  rt->st.pushed += n;
  return ATLAS_OK;
}

int atlas_rt_pump(atlas_rt_t rt, void* stream, int32_t max_tasks, atlas_rt_event* events, int32_t cap,
                  int32_t* n_events) {
  if (!rt || !n_events || cap < 0 || (cap > 0 && !events)) return ATLAS_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  EventSink sink{events, cap};
  const int SB = rt->o.search_block, OV = rt->o.search_overlap, TB = rt->o.track_block;
  int tasks = 0;
  while (max_tasks <= 0 || tasks < max_tasks) {
    const int64_t tail = std::max<int64_t>(0, rt->head - rt->cap);
    // tracking predictions whose block has already been overwritten are lost
    for (int c = 0; c < rt->C; ++c) {
      while (rt->tracking[c] && track_start(rt, c) < tail) {
        const double p = rt->pred[c];
        miss(rt, c);
        sink.add(make_event(ATLAS_RT_TRACK_LOST, c, track_start(rt, c), p, rt->misses[c]));
      }
    }
    // searching blocks that were overwritten are skipped
    if (rt->search_pos < tail) {
      sink.add(make_event(ATLAS_RT_SEARCH_SKIPPED, -1, rt->search_pos, 0.0, 0));
      rt->search_pos = tail;
    }
    std::vector<int> queue;
    for (int c = 0; c < rt->C; ++c)
      if (!rt->tracking[c]) queue.push_back(c);
    const bool search_ready = rt->search_pos + SB <= rt->head;
    if (search_ready && queue.empty()) {  // nothing to search: the block is passed over
      rt->search_pos += SB - OV;
      continue;
    }
    // the oldest pending transmission among the tracked codes whose block is complete
    int tc = -1;
    for (int c = 0; c < rt->C; ++c)
      if (rt->tracking[c] && track_start(rt, c) + TB <= rt->head && (tc < 0 || rt->pred[c] < rt->pred[tc])) tc = c;
    if (tc < 0 && !search_ready) break;
    const bool do_track = tc >= 0 && (!search_ready || rt->st.track_units <= rt->st.search_units);
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed_ms = [&] {
      return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    if (do_track) {
      const int64_t s = track_start(rt, tc);
      int n = 0;
      const int r = run_track(rt, st, tc, s, &n);
      if (r != ATLAS_OK) return r;
      rt->st.track_ms += elapsed_ms();
      rt->st.track_tasks += 1;
      rt->st.track_kernels += atlas_fsk_tracker_kernels(rt->trackers[rt->n_c[tc]]);
      rt->st.track_units += TB;
      if (n > 0) {
        const atlas_fsk_detection& d = rt->h_out[0];
        const double toa = (double)s + d.toa;
        rt->pred[tc] = toa + rt->period[tc];
        rt->misses[tc] = 0;
        atlas_rt_event e = make_event(ATLAS_RT_TRACK_DETECTION, tc, s, toa, 0);
        e.score = d.score;
        e.w_c = d.w_c;
        e.q = d.q;
        sink.add(e);
      } else {
        const double p = rt->pred[tc];
        miss(rt, tc);
        sink.add(make_event(ATLAS_RT_TRACK_MISS, tc, s, p, rt->misses[tc]));
      }
    } else {
      const int64_t s = rt->search_pos;
      int n = 0;
      const int r = run_block(rt, st, s, SB, queue, &n);
      if (r != ATLAS_OK) return r;
      rt->st.search_ms += elapsed_ms();
      rt->st.search_tasks += 1;
      rt->st.searched_samples += SB;
      rt->st.search_units += (int64_t)SB * (int64_t)queue.size();
      for (int i = 0; i < n; ++i) {  // ordered by (window, code): later windows re-anchor the prediction
        const atlas_fsk_detection& d = rt->h_out[i];
        const double toa = (double)s + d.toa;
        rt->tracking[d.code] = 1;
        rt->pred[d.code] = toa + rt->period[d.code];
        rt->misses[d.code] = 0;
        atlas_rt_event e = make_event(ATLAS_RT_SEARCH_DETECTION, d.code, s, toa, 0);
        e.score = d.score;
        e.w_c = d.w_c;
        e.q = d.q;
        sink.add(e);
      }
      rt->search_pos += SB - OV;
    }
    ++tasks;
  }
  rt->st.events += sink.n;
  *n_events = sink.n;
  return ATLAS_OK;
}

int atlas_rt_get_stats(atlas_rt_t rt, atlas_rt_stats* out) {
  if (!rt || !out) return ATLAS_ERR_INVALID_ARG;
  *out = rt->st;
  out->searching = out->tracking = 0;
  for (int c = 0; c < rt->C; ++c) (rt->tracking[c] ? out->tracking : out->searching) += 1;
  return ATLAS_OK;
}

const char* atlas_rt_last_error(atlas_rt_t rt) { return rt ? rt->last_error.c_str() : ""; }

void atlas_rt_destroy(atlas_rt_t rt) { free_rt(rt); }

}  // extern "C"
