// Schedule choice of the potential apply (see conv_impl.cuh): shared by the
// translation units of the three element types.
#pragma once

#include <string>

namespace bae {

// Three schedules compute the same transforms: five separate passes, the
// five passes with a second launch geometry (narrower column blocks, or the
// three-level transform plan), or the k and j passes fused per plane (where
// the plane fits in shared memory or a cluster). Which is faster depends on
// the precision, N and the batch size (the fused kernels run one 200 KB CTA
// per SM, fewer CTAs in flight). The first apply for a given (element type,
// N, batch size) outside a graph capture times every runnable schedule on
// the real data and keeps the fastest; the choices persist in the JSON file
// named by BAE_TUNE_FILE if set. BAE_CONV_PLANE=0/1/2/3 forces a schedule
// (the Sched values).

// SCHED_PASSES_ALT: the five passes with the variant-1 launch geometry
// (float32: half-width column blocks at N = 128, the three-level transform
// plan at N = 256; float64 at N = 128: the three-level transform plan;
// elsewhere the same as SCHED_PASSES).
// SCHED_PERSIST: the five passes as persistent kernels, each launched with
// at most the CTAs resident at once, which stride over the tiles of every
// right-hand side.
enum Sched { SCHED_PASSES = 0, SCHED_PLANE = 1, SCHED_PASSES_ALT = 2, SCHED_PERSIST = 3 };

// chosen schedule for a key "f32/N128/nb1", or -1 if none yet
int tune_lookup(const std::string& key);
void tune_store(const std::string& key, int sched);
// the schedule forced by set_forced_sched, else by BAE_CONV_PLANE=0..3; -1 if
// neither
int forced_sched();
// -1 (choose by timing), SCHED_PASSES, SCHED_PLANE, SCHED_PASSES_ALT or
// SCHED_PERSIST
void set_forced_sched(int sched);

}  // namespace bae
