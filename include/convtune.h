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
 * (tile width <= 256 floats), pitch and pointer alignment for the vector
 * width.  Returns CT_OK, CT_EINVAL (problem itself invalid) or CT_ECONFIG
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
 * back, all on `stream`, and returns after the stream has synchronised.
 * Pinned host memory gives the fastest copies; pageable memory works.
 */
int ct_conv2d_run_host(const float* in_host, long in_pitch, const float* filt, int fh, int fw,
                       float* out_host, long out_pitch, int out_h, int out_w,
                       const ct_config* c, void* stream);

/*
 * Device status word shared by the library's kernels (bit 0: a TMA tile wait
 * gave up; bit 1: a persistent-kernel wait gave up; bit 2: a work item was
 * out of range).  Reading synchronises the device; `clear` resets it.
 */
int ct_status_read(unsigned* bits, int clear);

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

#ifdef __cplusplus
}
#endif
#endif /* CONVTUNE_H */
