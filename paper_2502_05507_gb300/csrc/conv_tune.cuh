// Schedule choice of the potential apply (see conv_impl.cuh): shared by the
// translation units of the three element types.
#pragma once

#include <string>

namespace bae {

// Two schedules compute the same transforms: five separate passes, or the
// k and j passes fused per plane (where the plane fits in shared memory).
// Which is faster depends on the batch size (the fused kernels run one
// 200 KB CTA per SM, fewer CTAs in flight). The first apply for a given
// (element type, N, batch size) outside a graph capture times both on the
// real data and keeps the faster; the choices persist in the JSON file
// named by BAE_TUNE_FILE if set. BAE_CONV_PLANE=0/1 forces a schedule.

enum Sched { SCHED_PASSES = 0, SCHED_PLANE = 1 };

// chosen schedule for a key "f32/N128/nb1", or -1 if none yet
int tune_lookup(const std::string& key);
void tune_store(const std::string& key, int sched);
// the schedule forced by set_forced_sched, else by BAE_CONV_PLANE=0/1; -1 if
// neither
int forced_sched();
// -1 (choose by timing), SCHED_PASSES or SCHED_PLANE
void set_forced_sched(int sched);

}  // namespace bae
