// Internal launch interface of the fused 2^k cascade (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wd_common.cuh"
#include "wd_fwd.h"

namespace wdweno {

constexpr int CASCADE_MAX_LEVELS = 6;
// CTA width of the fused launch (all levels); a level's strips are
// CASCADE_THREADS - 9 output columns wide.
constexpr int CASCADE_THREADS = 128;

// One persistent launch over every tile of every level.  Tiles are numbered
// level by level (first[L] .. first[L + 1] - 1), within a level band-major:
// item = first[L] + (band * planes + plane) * strips + strip.  done[] holds,
// per level, band and plane, the count of finished strips (done_off[L] +
// band * planes + plane).
struct CascadeArgs {
  int levels;
  FwdArgs f[CASCADE_MAX_LEVELS];         // per level: input, output, sizes, band height
  MethodConsts k[CASCADE_MAX_LEVELS];    // per level: h halves from level to level
  int64_t strips[CASCADE_MAX_LEVELS];
  int64_t bands[CASCADE_MAX_LEVELS];
  int64_t first[CASCADE_MAX_LEVELS + 1];
  int64_t done_off[CASCADE_MAX_LEVELS];
  unsigned long long* head;  // next item
  unsigned int* done;        // finished-strip counters (all zeroed by the setup kernel)
  int64_t done_count;
};

cudaError_t launch_zoom2x_cascade(const CascadeArgs& c, int bmode, int in_t, int out_t,
                                  cudaStream_t stream);
cudaError_t fwd_wait_timeouts_cascade(unsigned int* count, bool reset);

}  // namespace wdweno
