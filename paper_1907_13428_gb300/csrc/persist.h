// Persistent executor of recorded launches (persist.cu): one cooperative kernel
// whose CTAs form instance groups; a group takes instances from a device-side
// queue and runs the bodies of each instance's recorded launches in order,
// with a bounded group barrier after each launch.
#pragma once
#include "internal.h"

namespace fde {

struct PersistLaunch {
  const unsigned char* cmds;  // device: recorded commands, kCmdBytes each
  const long long* off;       // device [count + 1]: first command of each instance
  const int* order;           // device [count]: queue order of the instances
  int count;                  // instances
  int groups, group_ctas;     // instance groups and CTAs per group (grid = groups * group_ctas)
  unsigned* bar;              // device [groups]: barrier arrival counters, zero at launch
  int* queue;                 // device [1]: next queue position, zero at launch
  int* slot;                  // device [groups]: instance claimed by each group
  long long* status;          // device [4]: FDE status, group, command index; zero at launch
  unsigned long long timeout_ns;  // limit of every barrier wait
  int stall_group;            // test hook: this group's first CTA skips its first arrival (-1: off)
  // lockstep schedule (every instance records the same number of launches):
  // step k runs launch k of every instance, its blocks spread over all CTAs
  int steps;                  // launches per instance (0: instance groups)
  const int* vstart;          // device [steps][count + 1]: prefix sums of the launches' grids
};

// Raise the persistent kernel's dynamic shared memory to `smem` and report how
// many of its CTAs fit on one SM.
cudaError_t persist_prepare(size_t smem, int* ctas_per_sm);
// Launch the persistent kernel cooperatively with pl.groups * pl.group_ctas CTAs
// (pl.steps > 0: the lockstep schedule, one group of all CTAs).
cudaError_t persist_run(const PersistLaunch& pl, size_t smem, cudaStream_t st);
// Issue the recorded commands (host copy) one by one as plain launches on st.
cudaError_t persist_replay(const unsigned char* cmds, long long n, cudaStream_t st);

}  // namespace fde
