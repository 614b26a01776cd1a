// Internal view of the platform table (energy counter, sensors, clocks).
#pragma once

#include "../../include/convtune.h"

namespace convtune {

// Snapshot of the current table (NVML-backed unless a caller installed one).
ct_platform_ops platform_ops();

// Monotonic seconds from the table's clock (host steady clock by default).
double platform_now(const ct_platform_ops& ops);

// Scoped clock lock: locks on construction (when mhz > 0) and resets in the
// destructor if the lock succeeded.  status() is the lock's result.
class ClockLock {
 public:
  ClockLock(const ct_platform_ops& ops, int mhz);
  ~ClockLock();
  int status() const { return status_; }
  bool locked() const { return locked_; }
  ClockLock(const ClockLock&) = delete;
  ClockLock& operator=(const ClockLock&) = delete;

 private:
  ct_platform_ops ops_;
  int status_ = 0;
  bool locked_ = false;
};

}  // namespace convtune
