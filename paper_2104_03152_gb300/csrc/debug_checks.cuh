// Debug build checks (compiled in with -DTCKS_DEBUG_CHECKS; the default build compiles them away).
//
// Host side: index and bounds assertions on the descriptor tables the batched launches build and on
// the job lists they come from (monotone first-job offsets, per-descriptor limb ranges that add up to
// the launch, context indices inside the table, job buffers that do not overlap another job's
// output). A failed assertion is an error return (TCKS_ERR_DEBUG_CHECK), never an abort.
//
// Device side: the descriptor-driven kernels check every index they derive from a descriptor (the
// context, the limb inside the descriptor's declared range, the prime inside the chain) before using
// it. A failed check sets a bit in the context's error word and skips the work item; the condition
// is the same for every thread of a CTA (and every CTA of a cluster), so a skip never leaves a
// barrier half-reached. The host reads the word after the batch and reports it.
#pragma once
#include <cstdint>

namespace tcks {

#ifdef TCKS_DEBUG_CHECKS
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif

// Bits of the error word.
enum : uint32_t {
  DBG_CTX_INDEX = 1u,   // descriptor names a context outside the launch's table
  DBG_LIMB_RANGE = 2u,  // work item outside its descriptor's declared limbs
  DBG_MOD_INDEX = 4u,   // prime index outside the context's chain
  DBG_NULL = 8u,        // null source or destination
};

#ifdef __CUDACC__
// True, with `bit` set in *word, when `ok` is false in a debug build; always false otherwise.
__device__ __forceinline__ bool dbg_fail(uint32_t* word, bool ok, uint32_t bit) {
  if (!kDebugChecks || ok) return false;
  if (word) atomicOr(word, bit);
  return true;
}
#endif

}  // namespace tcks
