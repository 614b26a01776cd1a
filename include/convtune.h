/*
 * convtune.h -- C ABI of libconvtune.so: energy-aware auto-tuning of an FP32
 * 2-D convolution on one GB300 (sm_103a).
 *
 * Source of the method: "Going green: optimizing GPUs for energy efficiency
 * through model-steered auto-tuning" (arXiv 2211.07260).
 *   - Energy of a run (Section III-A): E = integral of P dt, approximated by
 *     mean power x elapsed time.
 *   - Metrics and objectives (Section III-C): GFLOP/s, GFLOPs/W (= GFLOP/J);
 *     tuning for time, energy or efficiency; the SM clock as a tunable.
 *   - Power model and steering (Section IV-E, Eq. powercurve): fit
 *     P = min(P_max, P_idle + alpha f v^2) to a full-load kernel's power over
 *     the supported clocks, pick the clock minimising P/f and tune within
 *     +-10 % of it.
 * The convolution itself (block/tile sizes, halo staging, filter placement,
 * vector width) is the tuned workload, not a kernel printed in the paper.
 *
 * Conventions for every function below:
 *   - Return value: CT_OK (0) or a negative CT_E* status; ct_strerror()
 *     names it.  Nothing aborts the process; device kernels never trap.
 *   - Ownership: the caller owns every buffer it passes (host or device) and
 *     keeps it alive until the work using it has finished on its stream.  The
 *     library allocates only internal scratch (a device status word, staging
 *     buffers of the host-buffer entry point), released at unload.
 *   - Streams are cudaStream_t values passed as void*; NULL is the legacy
 *     default stream.  Launch functions are asynchronous and stream-ordered;
 *     they never synchronise unless stated.
 *   - Sizes are in elements unless a name ends in _bytes.
 */
#ifndef CONVTUNE_H
#define CONVTUNE_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
  CT_OK = 0,
  CT_EINVAL = -1,   /* bad argument: null pointer, size, pitch or alignment */
  CT_ENOTSUP = -2,  /* feature absent (NVML counter, TMA, driver entry point) */
  CT_EPERM = -3,    /* clock control not permitted (disabled, or denied)    */
  CT_ECUDA = -4,    /* a CUDA runtime / driver call failed                  */
  CT_ENOMEM = -5,   /* output capacity too small, or allocation failed      */
  CT_ETIMEOUT = -6, /* a bounded device wait gave up (see ct_status_read)   */
  CT_ECONFIG = -7,  /* configuration invalid for this problem or device     */
  CT_EIO = -8       /* results-cache file could not be read or written      */
};

/* Name of a status code (static string, never NULL). */
const char* ct_strerror(int status);

/* Library version, e.g. "convtune 0.1 sm_103a". */
const char* ct_version(void);

/* Name and text of the last CUDA error this thread saw inside the library
   (empty if none); the string lives until the thread's next library call. */
const char* ct_last_error(void);

/* ---- the tuned kernel --------------------------------------------------- */

/* Halo staging of the input tile a CTA needs. */
enum { CT_STAGE_DIRECT = 0, /* registers: global vector loads + warp shuffles */
       CT_STAGE_SMEM = 1,   /* shared memory, filled with cp.async            */
       CT_STAGE_TMA = 2 };  /* shared memory, one 2-D cp.async.bulk.tensor    */
/* Where the taps are read from. */
enum { CT_FILTER_SHARED = 0, /* copied to shared memory, read with LDS        */
       CT_FILTER_CONST = 1 };/* kernel parameter space (constant bank)        */

/* One point of the tuning space. */
typedef struct {
  int block_x;    /* threads per CTA in x: a multiple of 16, <= 1024        */
  int block_y;    /* threads per CTA in y: >= 1, block_x*block_y <= 1024    */
  int tile_x;     /* outputs per thread in x: 1, 2 or 4                     */
  int tile_y;     /* outputs per thread in y: 1, 2 or 4                     */
  int staging;    /* CT_STAGE_*                                             */
  int filter_mem; /* CT_FILTER_*                                            */
  int vec_width;  /* floats per global load / store: 1, 2 or 4              */
} ct_config;

/*
 * One correlation  out[y][x] = sum_{j<fh} sum_{i<fw} in[y+j][x+i]*filt[j][i]
 * for 0 <= y < out_h, 0 <= x < out_w (no filter flip).  `in` is the padded
 * input: out_h+fh-1 rows of in_pitch floats whose first out_w+fw-1 columns
 * are read (a "same" convolution of an out_h x out_w image takes
 * (fh-1)/2 and (fw-1)/2 zeros on each side, supplied by the caller).
 *   in, out : DEVICE pointers (16-byte aligned for vec_width 4 or TMA)
 *   filt    : HOST pointer to fh*fw floats, row-major; copied into the
 *             launch's parameters, so it may be reused as soon as the call
 *             returns
 *   fh, fw  : 1..32 with fh*fw <= 1024.  Square odd sides 1..17 run the
 *             specialised kernels; any other shape runs a generic kernel
 *             that honours only block_x / block_y of the configuration.
 */
typedef struct {
  const float* in;
  long in_pitch;
  const float* filt;
  int fh, fw;
  float* out;
  long out_pitch;
  int out_h, out_w;
} ct_problem;

/*
 * Check a configuration against a problem and the current device without
 * launching: block shape, register / shared-memory limits, TMA box limits
 * (tile height <= 256 rows; a tile wider than a 256-float box is staged as
 * one box per group of threads in x, each with its own halo), pitch and
 * pointer alignment for the vector width.  Returns CT_OK, CT_EINVAL (problem itself invalid) or CT_ECONFIG
 * (configuration pruned).  If `why` is non-NULL and why_cap > 0 a short
 * reason is written there (NUL-terminated).
 */
int ct_conv2d_check(const ct_problem* p, const ct_config* c, char* why, int why_cap);

/*
 * Launch the correlation with configuration c on `stream` (asynchronous).
 * Every configuration accumulates each output as one FP32 fmaf chain over
 * the taps in (j, i) lexicographic order, so all configurations return
 * bitwise-identical outputs.  Errors: CT_EINVAL, CT_ECONFIG, CT_ECUDA
 * (launch failure), CT_ENOTSUP (TMA staging without driver support).
 * Device-side failures (a bounded TMA wait giving up) set bits of the device
 * status word, read with ct_status_read().
 */
int ct_conv2d_run(const ct_problem* p, const ct_config* c, void* stream);

/*
 * The same correlation on HOST buffers (in: out_h+fh-1 rows of in_pitch
 * floats; out: out_h rows of out_pitch floats).  The library copies the
 * input to internal device buffers, runs the kernel and copies the result
 * back, and returns when the result is in `out`.  Work starts after the
 * caller's earlier work on `stream`; problems of 512 rows or more are split
 * into row bands (ct_conv2d_host_bands_default) whose input copies, kernels
 * and output copies overlap on library streams (results are identical to
 * one launch).  Pinned host memory gives the
 * fastest, overlapping copies; pageable memory works.
 */
int ct_conv2d_run_host(const float* in_host, long in_pitch, const float* filt, int fh, int fw,
                       float* out_host, long out_pitch, int out_h, int out_w,
                       const ct_config* c, void* stream);

/*
 * ct_conv2d_run_host that returns once the work is enqueued: the copies in,
 * the kernels and the copies out run on library streams, ordered after the
 * earlier host-buffer calls of this device (not after any caller stream:
 * `in` must hold its data at the call).  ct_conv2d_host_wait returns when
 * every earlier call's output is in its `out`; until then `in` must stay
 * allocated and unmodified and `out` allocated and unread.  The taps are
 * taken at the call.  The library keeps two sets of device buffers and
 * alternates them between calls, so a call's copies in overlap the previous
 * call's kernels and copies out (a stream of images keeps the host link
 * busy in both directions); each call is split into two row bands (one
 * below 512 rows).  With pageable host memory the copies may block
 * the calling thread.  Same arguments and errors as ct_conv2d_run_host;
 * errors found while enqueueing wait for the library's streams before
 * returning.  (Not in the paper: host-side pipelining.)
 */
int ct_conv2d_run_host_async(const float* in_host, long in_pitch, const float* filt, int fh,
                             int fw, float* out_host, long out_pitch, int out_h, int out_w,
                             const ct_config* c);
/* Wait for every earlier ct_conv2d_run_host_async call of the current
   device; returns the first CUDA error seen by them (CT_ECUDA) or CT_OK. */
int ct_conv2d_host_wait(void);

/*
 * ct_conv2d_run_host with the row bands given by the caller: band b covers
 * band_rows[b] output rows, in order from row 0 (band_rows[b] >= 1, their sum
 * == out_h, 1 <= n_bands <= 64; otherwise CT_EINVAL).  Each band is one
 * kernel launch whose input copy overlaps the previous band's kernel and the
 * output copy of the one before; results are identical to one launch for any
 * split.  ct_conv2d_run_host uses the split ct_conv2d_host_bands_default
 * returns.  (Pipelining of host copies: not in the paper, whose kernels read
 * device-resident inputs.)
 */
int ct_conv2d_run_host_bands(const float* in_host, long in_pitch, const float* filt, int fh,
                             int fw, float* out_host, long out_pitch, int out_h, int out_w,
                             const ct_config* c, const int* band_rows, int n_bands,
                             void* stream);

/*
 * The default split of out_h >= 1 output rows: an even split (sizes differ
 * by at most one row) into max(min(out_h / 256, 8), ceil(out_h / 512))
 * bands, at least 1 and at most 64.  Writes up to `cap` band sizes and the
 * count to *n_bands; CT_ENOMEM if cap is too small (the count is still
 * written), CT_EINVAL for out_h < 1 or a NULL n_bands.
 */
int ct_conv2d_host_bands_default(int out_h, int* band_rows, int cap, int* n_bands);

/*
 * Device status word shared by the library's kernels (bit 0: a TMA tile wait
 * gave up; bit 1: a persistent-kernel wait gave up; bit 2: a work item was
 * out of range).  Reading synchronises the device; `clear` resets it.
 */
int ct_status_read(unsigned* bits, int clear);

/*
 * Self-test of the bounded device waits: launches one CTA that waits on a
 * barrier phase nothing completes, gives up after spin_limit polls
 * (1 .. 2^24) and sets status bit 0 (as a TMA wait that gave up would); the
 * context stays usable.  Asynchronous on `stream`; read the bit with
 * ct_status_read().
 */
int ct_selftest_wait_timeout(unsigned spin_limit, void* stream);

/* Device facts used for rooflines (current device). */
typedef struct {
  int sm_count;
  int cc_major, cc_minor;
  int max_smem_optin_bytes;
  int l2_bytes;
  double sm_clock_max_mhz;   /* from NVML when available, else 0 */
  char name[96];
} ct_device_info;
int ct_device_info_get(ct_device_info* out);


/* ---- platform: energy counter, sensors, clock control ------------------- */

/*
 * Energy comes from the device's total-energy counter (NVML,
 * millijoules since driver load); power, SM clock, throttle reasons,
 * temperature and other compute processes are read beside it (the sensors
 * the paper's NVML observer records, Section III-B).  The default table is
 * backed by libnvidia-ml, loaded at run time; a caller (tests, simulations)
 * may install its own table.  Every function returns CT_OK or a CT_E*
 * status; a NULL member means "not available" (CT_ENOTSUP).
 *
 * Clock control (the paper's nvml_gr_clock tunable, Section III-C) changes
 * a device setting that outlives the process.  The NVML table refuses it
 * (CT_EPERM) unless the environment variable CONVTUNE_ALLOW_CLOCK_CONTROL
 * is "1"; when enabled, every lock is undone on return, on error and at exit.
 * Power limits (nvml_pwr_limit) are the same kind of setting: refused unless
 * CONVTUNE_ALLOW_POWER_CONTROL is "1", and restored to the device's default
 * on return, on error and at exit.
 */
enum { CT_UNIT_CONV = 0, CT_UNIT_FMA = 1, CT_UNIT_COPY = 2 };
/* Throttle-reason bits (same values as NVML's clocks-event reasons). */
enum { CT_THR_SW_POWER_CAP = 0x4, CT_THR_HW_SLOWDOWN = 0x8, CT_THR_SW_THERMAL = 0x20,
       CT_THR_HW_THERMAL = 0x40, CT_THR_HW_POWER_BRAKE = 0x80 };
typedef struct {
  void* ctx;
  int (*energy_mj)(void* ctx, unsigned long long* mj);
  int (*power_mw)(void* ctx, unsigned* mw);
  int (*sm_clock_mhz)(void* ctx, unsigned* mhz);
  int (*throttle_reasons)(void* ctx, unsigned long long* bits);
  int (*temperature_c)(void* ctx, unsigned* c);
  int (*other_processes)(void* ctx, int* n);
  int (*supported_sm_clocks)(void* ctx, int* mhz, int cap, int* n); /* descending */
  int (*lock_sm_clock)(void* ctx, int mhz);
  int (*reset_sm_clock)(void* ctx);
  double (*now_s)(void* ctx);  /* monotonic seconds; NULL: host steady clock */
  /* Simulation hook.  NULL: launches run on the GPU.  Otherwise the
     measurement calls this instead of launching: "run n launches of unit
     `kind` (CT_UNIT_*; cfg is the configuration for CT_UNIT_CONV, else NULL)
     and report their device time in *elapsed_ms". */
  int (*run_launches)(void* ctx, int kind, const ct_config* cfg, int n, double* elapsed_ms);
  /* Board power limit (the paper's nvml_pwr_limit tunable, Section IV-C),
     in mW: set, restore the device's default, and the allowed range. */
  int (*set_power_limit)(void* ctx, int mw);
  int (*reset_power_limit)(void* ctx);
  int (*power_limit_range)(void* ctx, int* min_mw, int* max_mw, int* default_mw);
} ct_platform_ops;

/* One reading of the platform's sensors (the observer record of Section
   III-B): NaN / 0 for sensors the table does not provide. */
typedef struct {
  double energy_j;        /* total-energy counter (since driver load)       */
  double power_w;         /* power reading (NVML: averaged over ~100 ms)    */
  double sm_clock_mhz;
  double temp_c;
  unsigned long long throttle_reasons;
  int other_processes;
} ct_sensors;
int ct_read_sensors(ct_sensors* out);

/* Install a platform table (copied); NULL restores the NVML table. */
int ct_set_platform_ops(const ct_platform_ops* ops);
/* CT_OK if the NVML table found libnvidia-ml and the current device. */
int ct_nvml_status(void);
/* Supported SM clocks of the current device, descending (MHz). */
int ct_supported_sm_clocks(int* mhz, int cap, int* n);
/* Lock / unlock the SM clock through the current table (see above). */
int ct_lock_sm_clock(int mhz);
int ct_reset_sm_clock(void);

/* ---- measurement of one point ------------------------------------------ */

typedef struct {
  double window_s;  /* energy window: mean power between two energy-counter
                       updates at least this far apart; <= 0 -> 1.0 s (the
                       paper's default observation time, Section III-B)   */
  double warmup_s;  /* continuous load before the window opens; < 0 -> 0.2 */
  double graph_ms;  /* target device time of one replayed CUDA graph of
                       back-to-back launches; <= 0 -> 2.0                  */
  int time_only;    /* 1: time the launches only, no energy window         */
  int time_reps;    /* graph replays timed when time_only; <= 0 -> 5       */
} ct_measure_options;

/* Record flags. */
enum { CT_REC_THROTTLED = 1,      /* a throttle reason was active           */
       CT_REC_COTENANT = 2,       /* another compute process was on the GPU */
       CT_REC_DEFAULT_CLOCKS = 4, /* clock requested but not locked         */
       CT_REC_INVALID = 8,        /* configuration pruned (not measured)    */
       CT_REC_CACHED = 16,        /* taken from the results cache           */
       CT_REC_NO_ENERGY = 32,     /* no energy counter: energy from power   */
       CT_REC_IDLE_GAPS = 64 };   /* the device idled inside the window     */

/* One measured point (the paper's observer record plus its metrics). */
typedef struct {
  ct_config cfg;
  int clock_mhz_req;       /* requested SM clock, 0 = default clocks        */
  double clock_mhz_meas;   /* median SM clock read during the window        */
  double t_s;              /* device time per launch (CUDA events)          */
  double energy_j;         /* energy per launch = mean power x t_s          */
  double power_w_mean;     /* energy-counter difference / window time       */
  double power_w_median;   /* median power reading in the window            */
  double energy_j_median_power; /* Section III-A estimate: median P x t_s   */
  double gflops;           /* useful GFLOP per launch / t_s                 */
  double gflops_per_j;     /* useful GFLOP per launch / energy_j            */
  double temp_c;           /* highest temperature read in the window        */
  double wall_s;           /* host seconds spent on this point              */
  int n_launches;          /* launches timed                                */
  int flags;               /* CT_REC_*                                      */
  double power_limit_w;    /* requested board power limit, 0 = the default  */
} ct_record;

/*
 * Measure one configuration: build a CUDA graph of back-to-back launches on
 * a private stream ordered after `stream`, warm up, then replay it while
 * reading the energy counter.  The energy window opens at one counter update
 * and closes at the first update at least window_s later, with the device
 * busy throughout; mean power over the window times the event-timed time per
 * launch gives the energy per launch.  Synchronises before returning.
 * Errors: as ct_conv2d_run; CT_ECONFIG leaves out->flags = CT_REC_INVALID.
 */
int ct_measure_conv(const ct_problem* p, const ct_config* c, const ct_measure_options* opt,
                    void* stream, ct_record* out);


/* ---- power model and steered clock range (Section IV-E) ----------------- */

/*
 * Eq. (powercurve): P*(f) = min(P_max, P_idle + alpha * f * v(f)^2), f in
 * GHz.  Without a voltage readout v(f) = 1 + beta * max(0, f - tau) (the
 * paper's estimate, read as continuous at the ridge point tau).
 * alpha: W/GHz (estimated v) or W/(GHz V^2) (measured v); beta: per GHz.
 */
typedef struct {
  double p_idle_w, alpha, beta, tau_mhz, p_max_w;
  int has_voltage;       /* 1: fitted with measured voltages               */
  double sse;            /* residual sum of squares of the kept samples    */
  int n_used;            /* samples kept (not throttled)                   */
  double f_lo_mhz;       /* lowest kept sample clock                       */
  double f_thr_mhz;      /* highest kept sample clock (before throttling)  */
  double f_opt_mhz;      /* clock minimising P*(f)/f on [f_lo, f_thr]      */
} ct_power_model;

/*
 * Fit the model to n samples (f_mhz[i], p_w[i]) with optional voltages and
 * throttle flags (flagged samples are dropped).  With voltages the fit is
 * linear least squares in x = f v^2; without, tau runs over the integer-MHz
 * grid of the kept clock range (needing two kept samples above it) and
 * (P_idle, alpha, beta >= 0) are fitted by Levenberg-Marquardt at each grid
 * point; the least residual wins, ties (1e-12 relative) keep the lower tau.
 * p_max_w <= 0 takes the largest measured power.  Needs >= 3 kept samples
 * (CT_EINVAL otherwise).  Host only; no GPU needed.
 */
int ct_fit_power_model(const double* f_mhz, const double* p_w, const double* v_or_null,
                       const int* throttled_or_null, int n, double p_max_w,
                       ct_power_model* out);
/* P*(f) of an estimated-voltage model at n clocks (MHz). */
int ct_model_power(const ct_power_model* m, const double* f_mhz, int n, double* p_w);
/* Clock minimising P*(f)/f over [f_lo, f_thr] (energy per cycle). */
int ct_optimal_clock(const ct_power_model* m, double* f_opt_mhz);
/*
 * Supported clocks c with (1-rel)*c0 <= c <= (1+rel)*c0, ascending, where c0
 * is the model optimum (center 0) or tau, the ridge point (center 1); an
 * empty window yields the nearest supported clock (ties: lower).  *n_out is
 * the count; CT_ENOMEM if it exceeds cap.
 */
int ct_pick_clock_range(const ct_power_model* m, const int* supported_mhz, int n_supported,
                        double rel_halfwidth, int center, int* out_mhz, int cap, int* n_out,
                        double* center_mhz);

/* ---- memory-aware energy model (Sections II and IV-F) ------------------- */

/*
 * Section IV-E estimates energy as P*(f)/f, i.e. run time ~ 1/f: right for
 * compute-bound kernels.  Section IV-F plans memory-dependent terms (the
 * estimate sometimes misses the measured optimum) and Section II recalls the
 * roofline energy model of Choi et al., where memory traffic costs energy
 * that compute cannot hide.  The paper gives no formula; this library reads
 * it as a run time with a clock-independent memory part,
 *
 *   t(f) = t_mem + c_core / f      (f in GHz; t_mem, c_core >= 0),
 *
 * fitted by non-negative linear least squares to a unit's (clock, time)
 * samples (throttled samples dropped), and energy per unit
 *
 *   E(f) = P*(f) * t(f),
 *
 * with P*(f) of Eq. powercurve fitted on the same unit's power samples.  For
 * t_mem = 0 this is the paper's estimate.  The stream-copy microbenchmark
 * (CT_UNIT_COPY) gives the memory-bound curve.
 */
typedef struct {
  double t_mem_s;        /* clock-independent time per unit (s)             */
  double c_core_s_ghz;   /* clock-bound time per unit at 1 GHz (s GHz)      */
  double sse;            /* residual sum of squares of the kept samples     */
  int n_used;            /* samples kept (not throttled)                    */
  double f_lo_mhz;       /* lowest kept sample clock                        */
  double f_thr_mhz;      /* highest kept sample clock                       */
} ct_time_model;

/*
 * Fit t(f) to n >= 2 samples (clocks in MHz > 0, times in s, throttled
 * optional): the unconstrained least-squares line in (1, 1/f) when both
 * coefficients are >= 0, else the better of the fits with t_mem = 0 or
 * c_core = 0 (each clamped at 0).  CT_EINVAL on bad input or fewer than two
 * kept samples.
 */
int ct_fit_time_model(const double* f_mhz, const double* t_s, const int* throttled_or_null,
                      int n, ct_time_model* out);
/* t(f) at n clocks (MHz). */
int ct_model_time(const ct_time_model* tm, const double* f_mhz, int n, double* t_s);
/*
 * Memory-aware optimum: the integer-MHz clock minimising P*(f) t(f) over
 * [max(pm.f_lo, tm.f_lo), min(pm.f_thr, tm.f_thr)] (ties: lower clock);
 * *e_opt_j (optional) receives E there.  The power model must be an
 * estimated-voltage fit (CT_EINVAL otherwise, or if the range holds no
 * integer clock).
 */
int ct_memory_aware_optimum(const ct_power_model* pm, const ct_time_model* tm,
                            double* f_opt_mhz, double* e_opt_j);
/*
 * Supported clocks within +-rel_halfwidth of center_mhz, ascending (the
 * +-10 % rule of Section IV-E around any centre); an empty window yields the
 * nearest supported clock (ties: lower).  CT_ENOMEM if *n_out exceeds cap.
 */
int ct_clock_range(double center_mhz, const int* supported_mhz, int n_supported,
                   double rel_halfwidth, int* out_mhz, int cap, int* n_out);

/* ---- tuning (Sections III-C and IV) ------------------------------------- */

enum { CT_OBJ_TIME = 0, CT_OBJ_ENERGY = 1, CT_OBJ_GFLOPS_PER_W = 2 };
/* Built-in spaces, in lexicographic order block_x, block_y, tile_x, tile_y,
   staging, filter_mem, vec_width:
   CT_SPACE_BASIC  block_x {16,32,64,128} x block_y {1,2,4,8} x tile_x, tile_y
                   {1,2,4} x staging {direct, smem}; constant filter, vector
                   width 4 (288 points);
   CT_SPACE_FULL   ... x staging {direct, smem, tma} x filter {shared, const}
                   x vector width {1,2,4} (2592 points). */
enum { CT_SPACE_BASIC = 0, CT_SPACE_FULL = 1 };
int ct_space(int which, ct_config* out, int cap, int* n);

typedef struct {
  int objective;                /* CT_OBJ_*                                 */
  ct_measure_options measure;   /* per-point measurement                    */
  const char* cache_path;       /* JSON-lines results cache; NULL: none     */
  double settle_s;              /* wait after each clock change             */
  int fallback_default_clocks;  /* 1: if locking is refused, measure once at
                                   default clocks (records flagged) instead
                                   of returning CT_EPERM                    */
} ct_tune_options;

/*
 * Exhaustive search of `space` (NULL: CT_SPACE_BASIC) x `clocks` (NULL or
 * n_clocks = 0: default clocks, no locking), clock-major so each clock is
 * locked once.  Invalid points are recorded with CT_REC_INVALID; cached
 * points (same device, problem, configuration, clock and window) are reused
 * and flagged CT_REC_CACHED; new points are appended to the cache as they are
 * measured, so an interrupted sweep resumes.  The clock is reset before
 * returning, on every path.  records[] receives n_space x max(1, n_clocks)
 * records in sweep order (CT_ENOMEM and *n_records = needed if cap is too
 * small; with fallback_default_clocks and a refused lock, one default-clock
 * pass of n_space records, flagged CT_REC_DEFAULT_CLOCKS); *best_index is the objective's optimum among valid records (ties:
 * shorter time, lower clock, lexicographically smaller configuration), or
 * -1.
 */
int ct_tune(const ct_problem* p, const ct_config* space, int n_space, const int* clocks_mhz,
            int n_clocks, const ct_tune_options* opt, void* stream, ct_record* records, int cap,
            int* n_records, int* best_index);

/*
 * Power capping instead of clock locking (Section IV-C compares the two):
 * exhaustive search of `space` x board power limits (mW, within the device's
 * range) at default clocks, limit-major, each limit set once and the
 * default restored before returning, on every path.  Records carry the limit
 * in power_limit_w (clock_mhz_req = 0); a power cap that lowered the clock
 * shows as CT_REC_THROTTLED.  Cache, records, capacity and selection as
 * ct_tune; with fallback_default_clocks a refused limit gives one pass at
 * the default limit flagged CT_REC_DEFAULT_CLOCKS.
 */
int ct_tune_power_limits(const ct_problem* p, const ct_config* space, int n_space,
                         const int* limits_mw, int n_limits, const ct_tune_options* opt,
                         void* stream, ct_record* records, int cap, int* n_records,
                         int* best_index);
/* The device's power-limit range and default (mW), from the platform table. */
int ct_power_limit_range(int* min_mw, int* max_mw, int* default_mw);

/* The selection rule of ct_tune over given records, optionally restricted to
   records whose requested clock is in clocks[] (n_clocks > 0). */
int ct_select_best(const ct_record* recs, int n, int objective, const int* clocks,
                   int n_clocks, int* best_index);


/* ---- microbenchmarks for the fit (Section IV-E) ------------------------- */

/*
 * CT_UNIT_FMA: a full-load FP32 kernel, 8 independent fmaf chains per
 * thread in registers (~1e9 FMAs per launch, 4 CTAs of 256 threads per SM;
 * *work = exact FLOP).  CT_UNIT_COPY: a 1 GiB float4 device-to-device copy
 * (*work = 2^31 bytes moved).  Their buffers are library scratch (2 GiB for
 * the copy), allocated on first use and freed by ct_microbench_release().
 */
int ct_microbench_launch(int which, void* stream, double* work);
/* Measure one microbenchmark at the current clocks (as ct_measure_conv). */
int ct_measure_microbench(int which, const ct_measure_options* opt, void* stream,
                          ct_record* out);
/*
 * Power samples for the fit: for each clock (locked in turn; NULL / 0
 * clocks: one sample at default clocks) measure the microbenchmark and
 * report the median SM clock, the mean power of the energy window (median
 * reading if the counter is absent) and whether it throttled (a throttle
 * reason, or the clock not held).  CT_EPERM if a lock is refused.
 */
int ct_measure_power_samples(int which, const int* clocks_mhz, int n_clocks,
                             const ct_measure_options* opt, void* stream, double* f_meas_mhz,
                             double* p_w, int* throttled, ct_record* recs_or_null);
int ct_microbench_release(void);

/* Result of the model-steered search. */
typedef struct {
  ct_power_model model;  /* the model the range is centred on (see below)   */
  double center_mhz;     /* its optimum                                     */
  int n_range;           /* clocks in the steered range                     */
  double fit_wall_s;     /* host seconds: microbenchmark sweeps + fits      */
  double tune_wall_s;    /* host seconds: the steered sweep                 */
  ct_power_model model_mem;  /* stream-copy power fit (CT_UNIT_COPY, union) */
  ct_time_model time_mem;    /* stream-copy time fit                        */
  double center_mem_mhz;     /* memory-aware optimum of the two             */
  int n_range_compute;       /* clocks around center_mhz (FMA model)        */
  int n_range_memory;        /* clocks around center_mem_mhz                */
} ct_steer_result;

/* which_bench value of ct_tune_steered: both models, union of their ranges */
enum { CT_STEER_UNION = 3 };

/*
 * Model-steered tuning (Section IV-E): sweep a microbenchmark over
 * fit_clocks (>= 3), fit, take the supported clocks (NULL: the platform's
 * list) within +-rel_halfwidth of the predicted optimum and run ct_tune over
 * that range only.  which_bench:
 *   CT_UNIT_FMA     the paper's model: Eq. powercurve on the FMA-dense
 *                   sweep, optimum of P*(f)/f (compute-bound kernels);
 *   CT_UNIT_COPY    the memory-aware model on the stream-copy sweep: power
 *                   and time fits, optimum of P*(f) t(f) (memory-bound
 *                   kernels); `model` / `center_mhz` repeat the copy fit;
 *   CT_STEER_UNION  both sweeps; the union of the two ranges (a kernel whose
 *                   boundness is unknown).
 * The fits use the requested clocks as f.  records / n_records / best_index
 * as ct_tune; range_out (optional) receives the tuned range.
 */
int ct_tune_steered(const ct_problem* p, const ct_config* space, int n_space,
                    const int* fit_clocks, int n_fit_clocks, const int* supported,
                    int n_supported, double rel_halfwidth, int which_bench,
                    const ct_tune_options* opt, void* stream, ct_steer_result* res,
                    int* range_out, int range_cap, ct_record* records, int cap, int* n_records,
                    int* best_index);


/* ---- batched correlation -------------------------------------------------- */

/*
 * Many correlations of uneven sizes and odd filter sides (1..17) behind one
 * host call and one CUDA-graph launch per batch.  A plan copies the taps and
 * an image table to the device (library scratch, freed by ct_batch_destroy)
 * and captures up to two graphs, both bitwise identical to ct_conv2d_run per
 * image (every tile uses the plain kernel's tap order):
 *
 *  - persistent: [work-counter reset + one persistent kernel per filter-side
 *    class] (sides 1-7, 9-11, 13-17: separate kernels so that each keeps its
 *    own register budget); images sorted by (filter side, size class).  CTAs
 *    of 256 threads, resident-occupancy x SM count of them per class kernel,
 *    take output tiles from a global atomic counter.  Tiles are 4 outputs
 *    wide per thread; per bucket (size class: output area < or >= 512^2;
 *    filter side) the block width and tile height come from ct_batch_tiles
 *    (0 or invalid entries: 32 x 8 threads, tile_y 2).
 *  - launches: one single-image kernel per image (compile-time filter side,
 *    taps in its parameter block), ordered by filter side and then output
 *    area (largest first), round-robin over 12 parallel graph branches; per bucket block_x x block_y threads and
 *    tile_y from the launch_* fields of ct_batch_tiles (0: 16 x 8, tile_y 4),
 *    TMA staging where the input allows it.  Captured for batches of at most
 *    CT_BATCH_LAUNCH_MAX_IMAGES images, unless the mode asked for is
 *    CT_BATCH_PERSISTENT; ct_batch_create then runs these launches once
 *    (writing every output, and returning after they finish) before it
 *    captures them, so that kernels are loaded outside the capture.
 *
 * ct_batch_run replays the batch's mode: ct_batch_tiles.mode, where
 * CT_BATCH_AUTO takes the launches graph when it exists and the images
 * average at least 65,536 outputs (each launch then fills a good part of the
 * GPU), else the persistent graph.  The plain comparison runs each image
 * with the persistent bucket's block and min(tile_y, 4), host-issued.
 */
enum { CT_BATCH_AUTO = 0, CT_BATCH_PERSISTENT = 1, CT_BATCH_LAUNCHES = 2 };
#define CT_BATCH_LAUNCH_MAX_IMAGES 1024
typedef struct {
  const float* in;    /* device, padded input: out_h+k-1 rows of in_pitch   */
  long in_pitch;
  const float* filt;  /* HOST, k*k taps row-major (copied at plan time)     */
  int k;              /* odd, 1..17                                         */
  float* out;         /* device                                             */
  long out_pitch;
  int out_h, out_w;   /* 0 x anything: skipped                              */
} ct_batch_item;

typedef struct {
  int block_x[2][18]; /* [size class][k]: 16, 32, 64 or 128, <= the class's CTA size
                         (block_y = CTA size / block_x)                      */
  int tile_y[2][18];  /* [size class][k]: 1, 2 or 4; also 8 for k <= 3     */
  int class_threads[3]; /* CTA size of the filter-side classes 1-7, 9-11,
                           13-17: 64, 128 or 256 (0: 256)                    */
  int claim_items[3];   /* work items (consecutive tiles) per claim of the
                           persistent CTAs, per class: 1..8 (0: 2, 1, 1)     */
  int launch_block_x[2][18]; /* launches graph, [size class][k]: 16, 32, 64,
                                128 (0: 16)                                   */
  int launch_block_y[2][18]; /* 1, 2, 4, 8 (0: 8); block_x x block_y <= 1024 */
  int launch_tile_y[2][18];  /* 1, 2, 4 (0: 4)                               */
  int mode;                  /* CT_BATCH_AUTO / _PERSISTENT / _LAUNCHES       */
} ct_batch_tiles;

typedef struct {
  int n_images;       /* non-empty images                                   */
  long long n_items;  /* output tiles                                       */
  int grid;           /* persistent CTAs, over all kernel launches          */
  long smem_bytes;    /* dynamic shared memory per CTA (largest launch)     */
  double flop;        /* useful FLOP per batch                              */
  double bytes;       /* algorithmic bytes per batch (inputs, outputs, taps) */
  int launches;       /* kernel launches per persistent run: one persistent
                         kernel per filter-side class present (sides 1-7,
                         9-11, 13-17), more when parameter blocks fill up    */
  int mode;           /* CT_BATCH_PERSISTENT or CT_BATCH_LAUNCHES: the graph
                         ct_batch_run replays                                */
  int has_launch_graph; /* 1: the launches graph was captured too            */
} ct_batch_stats;

typedef struct ct_batch ct_batch;  /* opaque plan */

int ct_batch_create(const ct_batch_item* items, int n, const ct_batch_tiles* tiles_or_null,
                    ct_batch** out);
/* Replay the captured batch (its mode's graph) on `stream` (asynchronous). */
int ct_batch_run(ct_batch* b, void* stream);
/* What ct_batch_run_mode and ct_measure_batch run: the batch's own mode,
   the plain comparison, the persistent graph, the launches graph
   (CT_ENOTSUP when it was not captured). */
enum { CT_BATCH_RUN_DEFAULT = 0, CT_BATCH_RUN_PLAIN = 1, CT_BATCH_RUN_PERSISTENT = 2,
       CT_BATCH_RUN_LAUNCHES = 3 };
int ct_batch_run_mode(ct_batch* b, int which, void* stream);
/* The comparison: one ct_conv2d_run per image (bucket configuration, taps
   from the parameter space), in table order, on `stream`. */
int ct_batch_run_plain(ct_batch* b, void* stream);
int ct_batch_info(const ct_batch* b, ct_batch_stats* out);
/* Waits for nothing; the caller must have synchronised work using b. */
int ct_batch_destroy(ct_batch* b);
/* Measure the batch as ct_measure_conv: `which` is a CT_BATCH_RUN_* value
   (graph replays for the graphs; host-issued launches, no graph, for the
   plain comparison). */
int ct_measure_batch(ct_batch* b, int which, const ct_measure_options* opt, void* stream,
                     ct_record* out);
/*
 * Per-bucket tile tuning: for every (size class, filter side) present,
 * block_x in {16, 32, 64, 128} (at most the class's CTA size) x tile_y in
 * {1, 2, 4} (and 8 for k <= 3) are measured and the objective's best is
 * kept.  Each candidate is measured on all the images of the bucket's
 * filter-side class as one batch, the class's other buckets at their current
 * tiles (one bucket after another): a class launch's staging buffers and
 * occupancy follow its largest tile.  `tiles` is read first -- its class CTA
 * sizes and claim sizes are kept and its valid tiles are the starting point
 * -- then receives the result.  records (optional: 16 per bucket with
 * k <= 3, 12 per other bucket at most) receive the measurements.
 */
int ct_batch_tune(const ct_batch_item* items, int n, int objective,
                  const ct_measure_options* opt, void* stream, ct_batch_tiles* tiles,
                  ct_record* records, int cap, int* n_records);
/*
 * Per-bucket tuning of the launches graph: for every (size class, filter
 * side) present, nine single-image configurations (block_x, block_y,
 * tile_y) in {(16,8,4), (32,4,4), (32,2,4), (16,4,4), (64,2,4), (32,8,2),
 * (32,4,2), (64,4,2), (128,2,2)} are measured, each as a launches graph of
 * the bucket's images, and the objective's best goes to the launch_* fields
 * of `tiles` (its other fields are kept).  records (optional: 9 per bucket)
 * receive the measurements, with the configuration the bucket's first image
 * ran (TMA staging, or its fallback).
 */
int ct_batch_tune_launches(const ct_batch_item* items, int n, int objective,
                           const ct_measure_options* opt, void* stream, ct_batch_tiles* tiles,
                           ct_record* records, int cap, int* n_records);


/* ---- batched correlation that allocates nothing -------------------------- */

/*
 * The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory (code running where a framework or memory
 * pool owns the GPU's memory, or under a rule against cudaMalloc once
 * serving has started, since an allocation can synchronise the device or
 * fail under memory pressure).
 *
 * It runs the same persistent batched kernel as ct_batch_run on the same
 * caller-owned inputs and outputs, but every piece of scratch it needs (work
 * counters, status word, image table, padded taps) lives in one fixed array
 * compiled into the library (about 373 KB, held on every GPU that loads the
 * library until the process exits).  Limit: n <= 256 images (filter sides
 * 1..17, odd); larger n returns CT_EINVAL and ct_last_error() says why.  No
 * cudaMalloc, cudaFree or other allocating routine is called.  The image
 * table and the taps (read from `filt`, host) go to the device as one copy
 * on `stream` from a per-thread host block in pageable memory; the runtime
 * stages such a copy before it returns and may first wait for work already
 * queued on `stream`, so the call can block until that work is done.  It
 * does not wait for its own kernels (inputs and outputs must stay alive
 * until the work completes).
 *
 * The first call on a device resolves the array's device address and raises
 * the kernel's shared-memory limit; make that first call before any stream
 * capture.  Every call reuses the same array (its contents are those of the
 * last call; the work counters are cleared each call), so calls whose work
 * overlaps on the GPU -- different streams, or different host threads --
 * race: serialise them on one stream.
 */
int ct_batch_run_noalloc(const ct_batch_item* items, int n, const ct_batch_tiles* tiles_or_null,
                         void* stream);
/*
 * The status word of the no-allocation scratch, also without allocating:
 * error bits the batched kernels raised in ct_batch_run_noalloc calls
 * (bit 2, as in ct_status_read: a work item outside its image, or a filter
 * side the launch's kernel does not hold).  The word is zero when the library loads
 * and keeps its bits across calls until this function clears it (clear != 0).
 * Reads on `stream` and waits for it, so the bits cover every call enqueued
 * there before; *bits receives the word.
 */
int ct_batch_noalloc_status(unsigned* bits, int clear, void* stream);


/* ---- request server with continuous batching ---------------------------- */

/*
 * Requests (host input, host taps, host output buffer) are submitted at any
 * time from any thread.  A worker thread admits them in arrival order while
 * a device-resident pool (allocated at creation, at most 90 % of the free
 * device memory) has room for their buffers, and dispatches admitted
 * requests as batches on up to n_streams streams at once: copy in, the
 * persistent batched kernels (one per filter-side class present; or, with
 * `plain`, one plain launch per request), copy out.  A batch leaves when it
 * is full, when no batch is in flight, or when its oldest request has
 * waited max_wait_s; requests that arrive while others run join the next
 * batch.  Results are bitwise equal to a request served alone.  Latency =
 * submission to completion seen by the worker.  Host buffers must stay
 * valid until the request completes.  Creation also loads every kernel the
 * worker can launch (kernel code is otherwise loaded on first use, which
 * would stall the worker with requests queued behind it).
 */
typedef struct {
  int n_streams;         /* batches in flight at once, 1..64                */
  int max_batch;         /* requests per batch, 1..4096                     */
  long long pool_bytes;  /* device pool for request buffers                 */
  double max_wait_s;     /* batching delay bound                            */
  int plain;             /* 1: one plain kernel per request (comparison)    */
  int use_tiles;         /* 1: per-bucket tiles from `tiles`                */
  ct_batch_tiles tiles;
  int trace_cap;         /* > 0: keep a timeline of the last trace_cap
                            batches (ct_server_trace_get); 0: none           */
} ct_server_options;

/* One batch of the worker's timeline (host steady-clock seconds). */
typedef struct {
  double t_dispatch;     /* the worker took the batch                       */
  double dispatch_s;     /* host time enqueueing it: copies, plan, launches */
  double plan_s;         /* of which: image table and launch plan           */
  double t_done;         /* the worker saw its completion event             */
  double oldest_wait_s;  /* its oldest request: submission to t_dispatch    */
  double loop_gap_s;     /* longest pause between two worker iterations
                            since the previous batch was taken              */
  int n_requests;
  int slot;              /* stream slot it ran on                           */
  int queued;            /* requests waiting for admission at t_dispatch    */
  int busy_slots;        /* other batches in flight at t_dispatch           */
  double h2d_ms;         /* device time (CUDA events on the batch's stream):
                            input copies                                     */
  double kernels_ms;     /* the batch's kernels                             */
  double d2h_ms;         /* output copies                                   */
  double bytes_in, bytes_out;  /* copied in / out                            */
} ct_server_trace_entry;

typedef struct {
  long long submitted, completed, rejected;
  double p50_s, p99_s, mean_s, max_s;  /* request latency                   */
  double wall_s;         /* creation or last reset to the last completion   */
  double flop;           /* useful FLOP of completed requests               */
  double energy_j;       /* energy-counter difference over the same span    */
  long long batches;
  double mean_batch;     /* requests per batch                              */
  long long pool_used_bytes;
} ct_server_stats;

typedef struct ct_server ct_server;

int ct_server_create(const ct_server_options* opt, ct_server** out);
/* Queue one request (k odd, 1..17); CT_ENOMEM if it can never fit the pool. */
int ct_server_submit(ct_server* sv, const float* in_host, long in_pitch, const float* filt, int k,
                     float* out_host, long out_pitch, int out_h, int out_w, long long* id);
/* Wait for one request (CT_ETIMEOUT on timeout); returns its status and
   releases its record.  latency_s may be NULL. */
int ct_server_wait(ct_server* sv, long long id, double timeout_s, double* latency_s);
/* Wait for every submitted request; releases their records. */
int ct_server_drain(ct_server* sv, double timeout_s);
/* Statistics since creation or the last reset (reset = 1 starts a new span). */
int ct_server_stats_get(ct_server* sv, int reset, ct_server_stats* out);
/* Finish every queued request, stop the worker and free the server. */
int ct_server_destroy(ct_server* sv);
/*
 * The timeline of the last completed batches (at most trace_cap, oldest
 * first): *n receives the count; CT_ENOMEM if it exceeds cap (the count is
 * still written); CT_ENOTSUP if the server keeps no timeline.  A diagnostic:
 * where a request's latency went (waiting for admission or a free slot,
 * enqueueing on the worker, device and copies, pauses of the worker).
 */
int ct_server_trace_get(ct_server* sv, ct_server_trace_entry* out, int cap, int* n);


/* ---- analyses of tuning records (Sections IV-A, IV-B) ------------------- */

/*
 * The five tuning methods compared in Section IV-A, over records of a
 * configuration x clock sweep (invalid records ignored): out[0] race-to-idle
 * (fastest point), out[1] least energy at the highest clock, out[2] the
 * fastest configuration at the highest clock then its least-energy clock,
 * out[3] the least-energy configuration at the base clock (the sampled clock
 * nearest base_clock_mhz) then its least-energy clock, out[4] global least
 * energy.  Indices into recs; ties as ct_select_best.
 */
int ct_tuning_methods(const ct_record* recs, int n, int base_clock_mhz, int out[5]);
/* Pareto front of (GFLOP/s, GFLOP/J), both maximised: indices of records no
   other record dominates, by GFLOP/s descending (ties: GFLOP/J, index). */
int ct_pareto_front(const ct_record* recs, int n, int* out_idx, int cap, int* n_out);
/*
 * Proportion of PageRank centrality (Section IV-B): nodes are the records;
 * two are neighbours when they differ in exactly one parameter (the seven
 * configuration fields and the clock); an edge leads to each neighbour of
 * strictly better fitness (time or energy); PageRank with the given damping
 * (0.85 in common use), walkers at minima restarting uniformly.  For each
 * p >= 1, out_prop = centrality of minima with fitness <= p * optimum over
 * centrality of all minima.
 */
int ct_centrality(const ct_record* recs, int n, int objective, double damping, const double* ps,
                  int n_p, double* out_prop);

#ifdef __cplusplus
}
#endif
#endif /* CONVTUNE_H */
