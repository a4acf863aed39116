// The persistent batch engine (persist.cu): host-side entry points used by
// the batched API (batched.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace rqk {

// Everything a launch of the persistent kernel needs, prepared once.
struct PersistLaunch {
  void *params;          // the kernel's parameter block (host copy)
  size_t param_bytes;
  void *zero_base;       // device region zeroed before every launch (counters, control blocks)
  size_t zero_bytes;
  int grid, smem;
  long long items;       // work items per launch
};

// Device workspace of the persistent engine for these problems and options,
// or 0 when the engine does not support them (precision other than FP64 and
// BF16x3, l > 128, n > 6000, given pivots, a truncation, BRQLP).
size_t persist_ws_bytes(const rqlp_problem *probs, int count, const rqlp_opts *o);

// Plans the batch (work items in list-schedule order, tensor maps, buffers)
// into the workspace, uploads the tables (synchronous copies: call outside a
// stream capture) and fills *out; d_status[i] receives problem i's status.
int persist_setup(const rqlp_problem *probs, int count, const rqlp_opts *o, void *ws,
                  size_t ws_bytes, int32_t *d_status, PersistLaunch *out);

// Enqueues one launch (the zeroing and the kernel) on st; capturable.
int persist_enqueue(const PersistLaunch &pl, cudaStream_t st);

// Per stage kind (16 slots, kinds 1..10 used) of the last launch: the time
// CTAs spent running items and waiting for them (dispatch and dependency
// waits), summed over CTAs, and the items that ran.
int persist_stats(const PersistLaunch &pl, cudaStream_t st, double *busy_us, double *wait_us,
                  int64_t *items);

void persist_release(PersistLaunch *pl);

}  // namespace rqk
