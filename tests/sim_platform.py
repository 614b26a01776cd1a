"""A simulated GPU behind the library's platform table (CPU tests).

Time advances only when the library "runs" launches through the table's
run_launches hook.  By default power follows Eq. (powercurve) of the paper
with known parameters (times a per-configuration utilisation), a launch
takes t_base(cfg) * f_max / f, and the total-energy counter is updated every
``period`` simulated seconds with the exact integral of power, in whole
millijoules -- the behaviour of NVML's counter on the GPU machine (~10 Hz
updates).

Options that make the device differ from the model the library fits:

* ``truth="curved"``: voltage rises through a smooth knee of width ``knee``
  MHz around tau, with curvature ``gamma`` (per GHz^2) on top of the linear
  rise, and static power grows with voltage (``leak``); Eq. (powercurve) can
  then only approximate the device.
* ``sigma_p`` / ``sigma_t``: relative Gaussian jitter of the power and the
  duration of every simulated run of launches (``seed`` seeds it).
* ``mem_frac``: the share of a configuration's (and ``copy_mem_frac`` of the
  stream copy's) run time that does not scale with the SM clock (memory
  bound); ``p_mem`` adds clock-independent memory power while the copy runs.

Board power limits (``plimit=(min_w, max_w, default_w)``): under a limit the
device runs each load at the highest supported clock (at most the locked or
maximum one) whose power stays within it, the lowest clock if none does, and
reports the software power-cap throttle reason while that lowers the clock.
"""
import ctypes
import math
import random

from paper_2211_07260_gb300 import api


class SimGPU:
    def __init__(self, p_idle=180.0, alpha=420.0, beta=0.9, tau=1380.0, f_max=2070,
                 clocks=None, period=0.1, lock_status=api.CT_OK, energy_status=api.CT_OK,
                 reasons=0, others=0, throttle_above=None, truth="powercurve", gamma=0.0,
                 knee=0.0, leak=0.0, sigma_p=0.0, sigma_t=0.0, seed=None, mem_frac=0.0,
                 copy_mem_frac=0.0, p_mem=0.0, plimit=None, plimit_status=api.CT_OK):
        self.p_idle, self.alpha, self.beta, self.tau = p_idle, alpha, beta, tau
        self.truth, self.gamma, self.knee, self.leak = truth, gamma, knee, leak
        self.sigma_p, self.sigma_t = sigma_p, sigma_t
        self.rng = random.Random(seed)
        self.mem_frac, self.copy_mem_frac, self.p_mem = mem_frac, copy_mem_frac, p_mem
        self.plimit = plimit          # (min, max, default) W, or None: no limit control
        self.plimit_status = plimit_status
        self.limit = None             # active board power limit (W)
        self.limit_calls = []
        self.limit_resets = 0
        self.capped = False           # the last run's clock was lowered by the limit
        self.cur_f = None             # the last run's clock
        self.f_max = f_max
        self.clocks = clocks or list(range(2070, 899, -15))
        self.period = period
        self.lock_status = lock_status
        self.energy_status = energy_status
        self.reasons = reasons
        self.others = others
        self.throttle_above = throttle_above  # clock cap that locks above cannot hold
        self.t = 0.0
        self.e = 0.0          # exact energy (J)
        self.e_tick = 0.0     # energy at the last counter update (J)
        self.locked = None
        self.lock_calls = []
        self.reset_calls = 0
        self.launches = 0
        self.last_power = p_idle
        self._ops = self._make_ops()

    # -- model ---------------------------------------------------------------
    def clock(self):
        f = self.locked if self.locked else self.f_max
        if self.throttle_above and f > self.throttle_above:
            f = self.throttle_above
        return f

    def run_clock(self, kind, cfg):
        """Clock a load runs at: the requested one, lowered under a power limit."""
        f = self.clock()
        self.capped = False
        if self.limit is not None:
            util = self.util(kind, cfg)
            ok = [c for c in self.clocks if c <= f and self.power_at(c, util, kind) <= self.limit]
            g = max(ok) if ok else min(self.clocks)
            self.capped = g < f
            f = g
        self.cur_f = f
        return f

    def voltage(self, f):
        if self.truth == "powercurve":
            return 1.0 + self.beta * max(0.0, f - self.tau) / 1000.0
        # smooth knee (softplus of width `knee` MHz) plus curvature
        x = (f - self.tau) / self.knee if self.knee > 0 else None
        if x is None:
            d = max(0.0, f - self.tau) / 1000.0
        else:
            d = self.knee * (x + math.log1p(math.exp(-x)) if x > 0 else math.log1p(math.exp(x)))
            d /= 1000.0
        return 1.0 + self.beta * d + self.gamma * d * d

    def power_at(self, f, util=1.0, kind=None):
        v = self.voltage(f)
        static = self.p_idle * (1.0 + self.leak * (v - 1.0))
        p = static + util * self.alpha * (f / 1000.0) * v * v
        if kind == api.CT_UNIT_COPY:
            p += self.p_mem
        return p

    def duration(self, kind, cfg, f):
        """Run time of one launch at SM clock f: the clock-bound share scales
        as f_max / f, the memory-bound share does not."""
        m = self.copy_mem_frac if kind == api.CT_UNIT_COPY else (
            0.0 if kind == api.CT_UNIT_FMA else self.mem_frac)
        return self.t_base(kind, cfg) * ((1.0 - m) * self.f_max / f + m)

    @staticmethod
    def t_base(kind, cfg):
        if kind == api.CT_UNIT_FMA:
            return 1.5e-3
        if kind == api.CT_UNIT_COPY:
            return 0.4e-3
        return 1e-4 * (1.0 + 0.13 * ((cfg.block_x // 16) % 3) + 0.07 * cfg.tile_y
                       + 0.05 * ((cfg.block_y + cfg.tile_x) % 4) + 0.02 * cfg.staging)

    @staticmethod
    def util(kind, cfg):
        if kind != api.CT_UNIT_CONV:
            return 1.0 if kind == api.CT_UNIT_FMA else 0.7
        return 0.75 + 0.05 * (cfg.tile_x % 3) + 0.04 * cfg.filter_mem

    def advance(self, dt, p):
        """Run at power p for dt seconds, updating the counter at ticks."""
        t1 = self.t + dt
        k0 = math.floor(self.t / self.period)
        k1 = math.floor(t1 / self.period)
        if k1 > k0:
            self.e_tick = self.e + p * (k1 * self.period - self.t)
        self.e += p * dt
        self.t = t1
        self.last_power = p

    # -- table callbacks -----------------------------------------------------
    def _make_ops(self):
        def energy(ctx, out):
            if self.energy_status != api.CT_OK:
                return self.energy_status
            out[0] = int(self.e_tick * 1000.0)
            return 0

        def power(ctx, out):
            out[0] = int(self.last_power * 1000.0)
            return 0

        def clock(ctx, out):
            out[0] = int(self.cur_f if self.cur_f is not None else self.clock())
            return 0

        def reasons(ctx, out):
            out[0] = self.reasons | (api.CT_THR_SW_POWER_CAP if self.capped else 0)
            return 0

        def temp(ctx, out):
            out[0] = 55
            return 0

        def others(ctx, out):
            out[0] = self.others
            return 0

        def supported(ctx, buf, cap, n):
            n[0] = len(self.clocks)
            if len(self.clocks) > cap:
                return api.CT_ENOMEM
            for i, c in enumerate(self.clocks):
                buf[i] = c
            return 0

        def lock(ctx, mhz):
            self.lock_calls.append(mhz)
            if self.lock_status != api.CT_OK:
                return self.lock_status
            self.locked = mhz
            return 0

        def reset(ctx):
            self.reset_calls += 1
            self.locked = None
            return 0

        def now(ctx):
            return self.t

        def run(ctx, kind, cfgp, n, ms):
            cfg = cfgp.contents if cfgp else None
            f = self.run_clock(kind, cfg)
            dt = n * self.duration(kind, cfg, f)
            p = self.power_at(f, self.util(kind, cfg), kind)
            if self.sigma_t:
                dt *= 1.0 + self.sigma_t * self.rng.gauss(0.0, 1.0)
            if self.sigma_p:
                p *= 1.0 + self.sigma_p * self.rng.gauss(0.0, 1.0)
            self.advance(dt, p)
            self.launches += n
            ms[0] = dt * 1e3
            return 0

        def set_limit(ctx, mw):
            self.limit_calls.append(mw)
            if self.plimit_status != api.CT_OK:
                return self.plimit_status
            self.limit = mw / 1000.0
            return 0

        def reset_limit(ctx):
            self.limit_resets += 1
            self.limit = None
            return 0

        def limit_range(ctx, lo, hi, de):
            lo[0], hi[0], de[0] = (int(w * 1000) for w in self.plimit)
            return 0

        ops = api.CtPlatformOps()
        ops.ctx = None
        ops.energy_mj = api._FN_ULL(energy)
        ops.power_mw = api._FN_UINT(power)
        ops.sm_clock_mhz = api._FN_UINT(clock)
        ops.throttle_reasons = api._FN_ULL(reasons)
        ops.temperature_c = api._FN_UINT(temp)
        ops.other_processes = api._FN_INTP(others)
        ops.supported_sm_clocks = api._FN_CLOCKS(supported)
        ops.lock_sm_clock = api._FN_LOCK(lock)
        ops.reset_sm_clock = api._FN_RESET(reset)
        ops.now_s = api._FN_NOW(now)
        ops.run_launches = api._FN_RUN(run)
        keep = [energy, power, clock, reasons, temp, others, supported, lock, reset, now, run]
        if self.plimit is not None:
            ops.set_power_limit = api._FN_LOCK(set_limit)
            ops.reset_power_limit = api._FN_RESET(reset_limit)
            ops.power_limit_range = api._FN_PLRANGE(limit_range)
            keep += [set_limit, reset_limit, limit_range]
        self._keep = tuple(keep)
        return ops

    def install(self):
        api.set_platform_ops(self._ops)
        return self

    @staticmethod
    def uninstall():
        api.set_platform_ops(None)

    # -- truth for the tests -------------------------------------------------
    def energy_per_launch(self, kind, cfg, f):
        """Noise-free energy of one launch at SM clock f (the truth)."""
        return self.power_at(f, self.util(kind, cfg), kind) * self.duration(kind, cfg, f)


class FakeBuffers:
    """Stand-ins for device buffers (the simulation never dereferences them)."""

    def __init__(self, out_h=512, out_w=512, k=7):
        self.out_h, self.out_w, self.k = out_h, out_w, k
        self.in_pitch = (out_w + k - 1 + 3) // 4 * 4
        self.out_pitch = out_w
        import numpy as np
        self.filt = np.full((k, k), 1.0 / (k * k), np.float32)
        self.inp = 0x100000
        self.out = 0x900000

    def args(self):
        return (self.inp, self.filt, self.out, self.out_h, self.out_w)
