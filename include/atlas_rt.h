/*
 * atlas_rt.h -- continuous ingest and the high-level scheduler (Section 2.2)
 * on top of the FSK search (atlas_fsk.h).
 *
 * Samples arrive as int16 (I, Q) pairs and are appended to a cyclic buffer in
 * device memory (Section 2: the receiver's samples go to a circular buffer
 * that allows processing delays of seconds).  The scheduler repeatedly picks
 * one task and runs it to completion (Section 2.2):
 *
 *   searching task: a block of search_block samples (100 ms by default),
 *     correlated with every code of the searching queue; consecutive blocks
 *     overlap by search_overlap samples (10 ms) so that every transmission
 *     lies inside one block.  A detected code moves to the tracking queue with
 *     its next arrival predicted one transmission period later.
 *   tracking task: one code, a block of track_block samples (12 ms) centred on
 *     the predicted arrival of its oldest pending transmission.  A detection
 *     re-anchors the prediction on the measured arrival; a miss (no detection,
 *     or samples already overwritten in the buffer) advances the prediction by
 *     one period, and after max_misses consecutive misses the code returns to
 *     the searching queue.
 *
 * The scheduler gives both kinds of task half of the work "in an amortized
 * sense" (Section 2.2).  Work is counted in deterministic units (samples x
 * codes of each task) rather than wall-clock time, so a given input always
 * produces the same task sequence.  When one kind has no ready task, the other
 * kind runs.  Tracking tasks go in order of predicted arrival.
 *
 * Every arrival time is absolute: samples from the first pushed sample.
 * Threading: one host thread per runtime; device work is ordered on the stream
 * passed to each call.  Errors as in atlas_acq.h.
 */
#ifndef ATLAS_RT_H_
#define ATLAS_RT_H_

#include <stdint.h>

#include "atlas_fsk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct atlas_rt* atlas_rt_t;

enum {
  ATLAS_RT_SEARCH_DETECTION = 0,  /* a searching task found the code */
  ATLAS_RT_TRACK_DETECTION = 1,   /* a tracking task found the predicted transmission */
  ATLAS_RT_TRACK_MISS = 2,        /* a tracking task found nothing (toa = the prediction) */
  ATLAS_RT_TRACK_LOST = 3,        /* the predicted block was overwritten before it was processed */
  ATLAS_RT_SEARCH_SKIPPED = 4     /* a searching block was overwritten before it was processed (code = -1) */
};

/* One scheduler outcome (48 bytes). */
typedef struct {
  int32_t kind;        /* ATLAS_RT_* */
  int32_t code;
  int64_t task_start;  /* absolute index of the task block's first sample */
  double  toa;         /* absolute arrival time in samples (the prediction for misses) */
  float   score;       /* as atlas_fsk_detection (0 for misses) */
  int32_t misses;      /* consecutive misses of the code after this task */
  double  w_c;         /* as atlas_fsk_detection */
  double  q;
} atlas_rt_event;

typedef struct {
  int64_t ring_samples;    /* cyclic buffer capacity in samples; default 16 s at fs */
  int32_t search_block;    /* default 0.1 s at fs */
  int32_t search_overlap;  /* default 0.01 s at fs */
  int32_t track_block;     /* default 0.012 s at fs */
  int32_t max_misses;      /* default 3 */
  int32_t capacity;        /* detection records per task; default 1024 */
  int32_t reserved[3];
} atlas_rt_opts;

typedef struct {
  int64_t pushed;          /* samples appended so far */
  int64_t search_tasks, track_tasks;
  int64_t searched_samples;  /* samples covered by searching blocks (overlaps counted twice) */
  int64_t search_units, track_units;  /* work units (samples x codes) of each kind */
  int64_t events;
  int64_t track_kernels;   /* kernel launches of the tracking tasks (their graphs' kernel nodes) */
  double  search_ms, track_ms;  /* host wall-clock time of the tasks of each kind, from launch to results */
  int32_t searching, tracking;  /* codes in each queue now */
  int32_t reserved;
} atlas_rt_stats;

void atlas_rt_default_opts(atlas_rt_opts* opts, double fs_hz);

/*
 * Create a runtime over an FSK context (borrowed: it must outlive the
 * runtime, and is used by the runtime alone while the runtime exists).
 *   period_samples  host, [n_codes] transmission period of each tag, samples (> 0)
 * Requires search_block >= search_overlap + 1, search_overlap >= the largest
 * support n_c (so that every transmission lies inside one searching block),
 * track_block >= the largest n_c, ring_samples >= search_block + track_block.
 * Allocates the cyclic buffer, a staging block and the result buffers.
 */
int atlas_rt_create(atlas_rt_t* out, atlas_fsk_t fsk, const double* period_samples, int32_t n_codes,
                    const atlas_rt_opts* opts);

/* Append n samples (host memory, [n][2] int16, read before the call returns)
 * to the cyclic buffer; the oldest samples are overwritten once it is full.
 * Stream-ordered. */
int atlas_rt_push(atlas_rt_t rt, void* stream, const int16_t* h_iq, int64_t n);

/* Run ready tasks, at most max_tasks (<= 0: until none is ready), appending
 * up to cap events to `events` (host); *n_events gets the number of events
 * produced (may exceed cap; only cap are written).  Synchronises `stream`
 * after every task (the next decision depends on its outcome). */
int atlas_rt_pump(atlas_rt_t rt, void* stream, int32_t max_tasks, atlas_rt_event* events, int32_t cap,
                  int32_t* n_events);

int atlas_rt_get_stats(atlas_rt_t rt, atlas_rt_stats* out);
const char* atlas_rt_last_error(atlas_rt_t rt);
void atlas_rt_destroy(atlas_rt_t rt);

#ifdef __cplusplus
}
#endif

#endif /* ATLAS_RT_H_ */
