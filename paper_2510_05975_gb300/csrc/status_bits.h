// status_bits.h -- bits of the device status word that kernels set (host and device).
#pragma once

#include <stdint.h>

namespace cng {

enum : uint32_t {
  ST_TIMEOUT = 1u,    // a bounded wait ran out
  ST_OVERFLOW = 2u,   // a fixed-capacity buffer would have overflowed
  ST_CERT = 4u,       // a row could not be certified even by the exact rescan
  ST_BOUNDS = 8u,     // an index failed its range check
  ST_SCREEN = 16u,    // screened score inconsistent with the stated exactness assumption
  ST_OVF_MERGE = 32u, // a merged candidate set exceeded its buffer
  ST_OVF_RUN = 64u,   // a run of near-tied distances longer than the FP64 re-sort buffer
};

}  // namespace cng
