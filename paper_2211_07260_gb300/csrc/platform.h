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

// Scoped board power limit: set on construction (when mw > 0), the device's
// default restored in the destructor if it was set.
class PowerLimit {
 public:
  PowerLimit(const ct_platform_ops& ops, int mw);
  ~PowerLimit();
  int status() const { return status_; }
  bool set() const { return set_; }
  PowerLimit(const PowerLimit&) = delete;
  PowerLimit& operator=(const PowerLimit&) = delete;

 private:
  ct_platform_ops ops_;
  int status_ = 0;
  bool set_ = false;
};

}  // namespace convtune
