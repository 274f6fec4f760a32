// check.cuh -- in-kernel bounds checks of the ZK_CHECK build.
//
// compute-sanitizer is not available where this library is tested on GPUs,
// so a build with -DZK_CHECK compiles checks of the invariants the kernels
// rely on at their gathers and scatters: scalars below r, bucket keys
// inside their job's bucket range, sorted-entry positions inside their
// bucket, NTT indices inside the vector.  A failed check sets a bit in a
// device flag word of its translation unit and skips the access; nothing
// traps.  zk_check_status reads and clears the flags.  In the normal build
// every check compiles to nothing.
#pragma once
#include <cstdint>

namespace zk {

// Flag bits.
constexpr uint32_t kCheckScalar = 1u << 0;   // a scalar >= r reached the MSM
constexpr uint32_t kCheckBucket = 1u << 1;   // a bucket key outside its job's range
constexpr uint32_t kCheckEntry = 1u << 2;    // a sorted-entry position outside its bucket
constexpr uint32_t kCheckNttIdx = 1u << 3;   // an NTT gather or scatter outside the vector

#ifdef ZK_CHECK
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

}  // namespace zk

// Per translation unit: the flag word and ZK_FAILED(cond, bit), which is
// true (and records the bit) when cond does not hold -- always false in the
// normal build.
#ifdef ZK_CHECK
#define ZK_CHECK_UNIT()                                                       \
    namespace {                                                               \
    __device__ uint32_t g_zk_check_flags;                                     \
    __device__ __forceinline__ bool zk_failed(bool ok, uint32_t bit) {        \
        if (!ok) atomicOr(&g_zk_check_flags, bit);                            \
        return !ok;                                                           \
    }                                                                         \
    }
#define ZK_FAILED(cond, bit) zk_failed((cond), (bit))
#else
#define ZK_CHECK_UNIT()
#define ZK_FAILED(cond, bit) false
#endif
