/*
 * A platform table for the library's clock-control tests: every call is
 * logged to a file (one line each) and nothing touches a GPU or NVML.
 * fake_install(path) installs it through ct_set_platform_ops().
 */
#include <stdio.h>
#include <string.h>

#include "convtune.h"

static FILE* g_log;
static int g_locked;

static void note(const char* what, int v) {
  if (!g_log) return;
  fprintf(g_log, "%s %d\n", what, v);
  fflush(g_log);
}
static int f_energy(void* c, unsigned long long* mj) { (void)c; *mj = 0; return CT_OK; }
static int f_power(void* c, unsigned* mw) { (void)c; *mw = 100000; return CT_OK; }
static int f_clock(void* c, unsigned* mhz) { (void)c; *mhz = g_locked ? (unsigned)g_locked : 2000u; return CT_OK; }
static int f_lock(void* c, int mhz) { (void)c; g_locked = mhz; note("lock", mhz); return CT_OK; }
static int f_reset(void* c) { (void)c; g_locked = 0; note("reset", 0); return CT_OK; }

int fake_install(const char* log_path) {
  ct_platform_ops ops;
  memset(&ops, 0, sizeof(ops));
  g_log = fopen(log_path, "a");
  ops.energy_mj = f_energy;
  ops.power_mw = f_power;
  ops.sm_clock_mhz = f_clock;
  ops.lock_sm_clock = f_lock;
  ops.reset_sm_clock = f_reset;
  return ct_set_platform_ops(&ops);
}
