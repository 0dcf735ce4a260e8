/*
 * adfft: the alpha-densified DFT on NVIDIA GB300 (sm_103a).
 *
 * For N samples x_n of a record of length T (t_n = nT/N, Eq. 3) and a dense
 * sampling factor alpha with M = alpha*N an integer, the library computes the
 * M output bins (Sec. 2, Eqs. 6-7, with the T/N scale of Eq. 2)
 *
 *     X_m = S * sum_{n=0}^{N-1} x_n * exp(-2*pi*i * m*n / M),   m = 0 .. M-1,
 *
 * whose bin interval is 1/(alpha*T).  S defaults to T/N with T = 1 (that is,
 * 1/N); adfft_plan_set_scale(plan, 1.0) gives Eq. 7 exactly as printed.  The
 * sign convention is W_M^{mn} = exp(-2 pi i m n / M) (Sec. 3).  For alpha > 1
 * this equals the length-M DFT of x zero-padded to M (Sec. 2); for alpha < 1 it
 * is the "one-way" transform of Sec. 2.
 *
 * Fast form (Sec. 3, Eqs. 9-15, written in the decimation-in-frequency order):
 * with g = gcd(M, N), P = M/g and q = N/g, bin m = P*k + r (k < g, r < P) is
 *     X_{Pk+r} = S * FFT_g( sum_{f<q} x_{n+g f} W_M^{r (n + g f)} )[k],
 * i.e. P twiddled length-g FFTs (q = 1 for integer alpha, which is the
 * "twiddle by W_M^{rn}, then alpha length-N FFTs" form).  Lengths g that are
 * not a power of two, or too large a fold q, use a chirp-z (Bluestein)
 * evaluation of the same sum.  Real input is packed two samples per complex
 * element and unpacked in the output epilogue.
 *
 * Conventions for every entry point:
 *   - Device buffers and the CUDA stream belong to the caller.  The plan owns
 *     its twiddle/chirp tables and any workspace; both live in device memory
 *     allocated by adfft_plan_create* and freed by adfft_plan_destroy.
 *   - Execution is stream-ordered and asynchronous; a plan may run on one
 *     stream at a time (calls on different streams that overlap race on the
 *     plan's workspace).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Data layout: input [batch][N] contiguous (real: float/double; complex:
 *     interleaved re,im); output [batch][M] complex, bins in natural order
 *     m = 0..M-1 (bins above M/2 are the negative frequencies).  Real input
 *     still yields all M bins.  Device pointers must be 16-byte aligned.
 *   - Every call returns ADFFT_OK (0) or a negative adfft_status; a call that
 *     fails launches nothing.  No C++ exception crosses this interface.
 *   - Failure injection for tests: the environment variable ADFFT_FAULT, read
 *     when a plan is created, makes that plan fail on purpose (unset: no
 *     effect).  "alloc:<k>": the k-th device allocation of the creation fails
 *     (the creation returns NULL, adfft_last_error() = ADFFT_ERR_OOM, nothing
 *     stays allocated); "launch": every launch of the plan fails (the calls
 *     return ADFFT_ERR_CUDA and launch nothing); "copy_skip:<s>": the fused
 *     kernel does not issue the input copy of signal s and gives up waiting for
 *     it after ~10 ms, so adfft_plan_sync_status reports ADFFT_ERR_TIMEOUT (the
 *     cluster concerned transforms no later signal; nothing faults or hangs).
 */
#ifndef ADFFT_H
#define ADFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADFFT_ABI_VERSION 1

typedef struct adfft_plan_s *adfft_plan_t;

/* Input element type; the output is complex of the same precision. */
typedef enum {
    ADFFT_R32 = 0,  /* real float32 input   -> complex64 (float2) output  */
    ADFFT_C64 = 1,  /* complex64 input      -> complex64 output           */
    ADFFT_R64 = 2,  /* real float64 input   -> complex128 (double2) output */
    ADFFT_C128 = 3  /* complex128 input     -> complex128 output          */
} adfft_dtype_t;

typedef enum {
    ADFFT_OK = 0,
    ADFFT_ERR_INVALID_ARG = -1,      /* NULL plan/pointer, N < 1, batch < 0, bad enum */
    ADFFT_ERR_INVALID_ALPHA = -2,    /* alpha not finite or <= 0, or alpha*N not an integer */
    ADFFT_ERR_UNSUPPORTED_SIZE = -3, /* sizes beyond what any kernel of the plan handles */
    ADFFT_ERR_MISALIGNED = -4,       /* a device pointer is not 16-byte aligned */
    ADFFT_ERR_OVERLAP = -5,          /* input and output ranges overlap (no in-place form) */
    ADFFT_ERR_CUDA = -6,             /* CUDA runtime or launch error */
    ADFFT_ERR_OOM = -7,              /* device allocation failed */
    ADFFT_ERR_TIMEOUT = -8,          /* a bounded device-side wait expired */
    ADFFT_ERR_NOT_SUPPORTED = -9     /* the plan's configuration lacks this operation */
} adfft_status_t;

/* Algorithm choice (adfft_plan_set_algorithm). */
typedef enum {
    ADFFT_ALGO_AUTO = 0,       /* the plan's own choice: the default rule below, or the autotuner's */
    ADFFT_ALGO_FOLD = 1,       /* P twiddled length-g FFTs in one fused pass (integer alpha: q = 1);
                                  where no single-pass shape fits, its two-pass variant */
    ADFFT_ALGO_BLUESTEIN = 2,  /* chirp-z: mn = (m^2 + n^2 - (m-n)^2)/2, convolution by FFT */
    ADFFT_ALGO_FOUR_STEP = 3   /* the fold form with each length-g FFT split g = A*B over two
                                  HBM passes (power-of-two g; plan workspace of batch*M complex) */
} adfft_algo_t;

/* Arithmetic form of the length-g FFT stages (adfft_plan_set_precision). */
typedef enum {
    ADFFT_PREC_NATIVE = 0,     /* FP32 for R32/C64 plans, FP64 for R64/C128 plans */
    ADFFT_PREC_FP16X2 = 1,     /* tensor-core radix-16 stages, fp16 hi+lo split operands (3 products),
                                  FP32 accumulate */
    ADFFT_PREC_BF16X3 = 2      /* tensor-core radix-16 stages, operands split into three bf16 parts
                                  (6 products), FP32 accumulate */
} adfft_precision_t;

/* Read-only description of a plan (adfft_plan_get_info). */
typedef struct {
    int64_t N;            /* samples per signal */
    int64_t M;            /* output bins per signal, M = alpha*N */
    int64_t batch;        /* signals (ragged plans: count) */
    int32_t dtype;        /* adfft_dtype_t */
    int32_t algo;         /* algorithm actually used (adfft_algo_t, never AUTO) */
    int64_t fft_len;      /* g: length of each sub-FFT (Bluestein: the padded length L) */
    int64_t residues;     /* P = M/g sub-FFTs per signal (Bluestein: output chunks) */
    int64_t fold;         /* q = N/g (Bluestein: 0) */
    int32_t cluster;      /* CTAs per signal sharing one thread-block cluster */
    int32_t passes;       /* HBM passes per forward transform (1 = fused single pass) */
    double scale;         /* S */
    int32_t staged;       /* 1 if the fused pass stages each signal through shared memory,
                             2 if its residues are exchanged by bulk push copies */
    int32_t tuned;        /* 1 if the launch shape came from the autotuner or its cache
                             (ragged plans: every shape class) */
    int32_t grid;         /* clusters the (first) kernel launches; each loops over signals */
    int32_t four_step_a;  /* four-step form: length A of the pass-1 transforms (fft_len = A*B) */
    int64_t out_bins;     /* output bins written per signal: M, or M/2 + 1 (half spectrum) */
} adfft_plan_info_t;

/* Output range (adfft_plan_set_output). */
typedef enum {
    ADFFT_OUTPUT_FULL = 0,     /* all M bins m = 0 .. M-1 (the default) */
    ADFFT_OUTPUT_HALF = 1      /* real input: bins m = 0 .. M/2 only ([batch][M/2 + 1] output) */
} adfft_output_t;

/*
 * Create a plan for `batch` signals of N samples and dense sampling factor
 * alpha (Eq. 6), M = alpha*N bins each.  alpha*N must be an integer to within
 * 1e-9*alpha*N (it is rounded to the nearest integer); alpha may be below 1.
 * Returns NULL on failure; adfft_last_error() then gives the reason.
 * Allocates the plan's tables (and workspace, if its algorithm needs one) on
 * the current CUDA device.
 */
adfft_plan_t adfft_plan_create(int64_t N, double alpha, int64_t batch, int dtype);

/* Same as adfft_plan_create with the bin count M given exactly (alpha = M/N). */
adfft_plan_t adfft_plan_create_bins(int64_t N, int64_t M, int64_t batch, int dtype);

/*
 * Ragged plan: `count` signals with their own N[i] and alpha[i] (each as in
 * adfft_plan_create), packed back to back: signal i occupies input elements
 * [in_off[i], in_off[i] + N[i]) and output bins [out_off[i], out_off[i] + M[i]),
 * offsets as returned by adfft_plan_offsets.  Signals are grouped into shape
 * classes of equal (N, M); each class is one persistent launch of the fused
 * kernel (its clusters loop over the class's signals through a device table of
 * offsets), and all class launches, forked over internal streams, are captured
 * into one CUDA graph at the first execute for a given buffer pair and
 * replayed by later executes.  Only ADFFT_R32 and ADFFT_C64 are accepted.
 */
adfft_plan_t adfft_plan_create_ragged(const int64_t *N, const double *alpha, int64_t count,
                                      int dtype);

/* Forward form of a ragged plan (adfft_plan_set_ragged_form). */
typedef enum {
    ADFFT_RAGGED_CLASSES = 0,  /* one persistent launch per shape class, all captured in one
                                  CUDA graph (forked over internal streams); the default */
    ADFFT_RAGGED_QUEUE = 1     /* one persistent kernel for the whole batch over a work queue
                                  of tiles (an option: slower on the 10000-signal mix) */
} adfft_ragged_form_t;

/*
 * Choose how a ragged plan's forward transform runs.  ADFFT_RAGGED_QUEUE: one persistent
 * kernel (as many CTAs as are resident) takes tiles from a queue in order: a "whole" tile
 * transforms signals whose residue FFTs fit one CTA's shared memory (up to 64 signals of a
 * class side by side); a longer signal is split into "fft" tiles (a group of its residues, the
 * sub-FFT results written to plan workspace) followed in the queue by "unpack" tiles (a
 * range of its output bins, gathered from that workspace once its fft tiles are counted,
 * queued about one wave of resident CTAs after them; the wait is bounded).  The execute is a memset of the queue counters plus that launch,
 * captured in a CUDA graph like the other form.  Served when every shape class is FP32 or
 * complex64 with even N and M for real input (packed) and a fold of at most 64 blocks onto
 * a power-of-two sub-FFT of at most 4096 points dividing its length and bin count; plan
 * workspace = 8 bytes per packed bin of the split signals (those whose residue FFTs exceed
 * 4096 points).  ADFFT_ERR_NOT_SUPPORTED for plans it cannot serve or non-ragged plans.
 * The adjoint always uses the class graph.
 */
int adfft_plan_set_ragged_form(adfft_plan_t plan, int form);

/*
 * Inspection of the queue form: the tile list that ADFFT_RAGGED_QUEUE runs for a ragged batch
 * of these shapes (N[i], alpha[i], as for adfft_plan_create_ragged), computed on the host from
 * the shapes alone (no device, no CUDA call).  Shape classes are the distinct (N, M) in
 * increasing order, as the ragged plan forms them.  lag: fft tiles between a split signal's
 * last fft tile and its first unpack tile (a plan uses its resident CTA count, e.g. 608).
 * Each tile is 5 int32 at tiles[5 i ..]: kind (0 whole, 1 fft, 2 unpack), class, then
 *   whole:  index of its first signal in whole[], 0, number of signals;
 *   fft:    signal, first residue, number of residues;
 *   unpack: signal, first leader bin, end leader bin (exclusive).
 * whole[] lists the signals of the whole tiles, tile after tile.  *ntiles and *nwhole receive
 * the counts; with tiles / whole NULL only the counts are written.  ADFFT_ERR_INVALID_ARG for
 * a capacity below the count, ADFFT_ERR_NOT_SUPPORTED for shapes the queue form cannot
 * serve (the same condition as adfft_plan_set_ragged_form), ADFFT_ERR_INVALID_ALPHA as for
 * plan creation.  The paper's method, generalised per signal (Sec. 3, Eqs. 10-13), is what
 * the tiles compute; the layout itself is this library's scheduling.
 */
int adfft_ragged_queue_layout(const int64_t *N, const double *alpha, int64_t count, int dtype, int32_t lag,
                              int32_t *tiles, int64_t tile_capacity, int64_t *ntiles, int64_t *whole,
                              int64_t whole_capacity, int64_t *nwhole);

/* Packed offsets of a ragged plan (arrays of count+1 entries; either may be NULL).
 * For a uniform plan: in_off[i] = i*N, out_off[i] = i*M. */
int adfft_plan_offsets(adfft_plan_t plan, int64_t *in_off, int64_t *out_off);

/* Status code of the last failed adfft_plan_create* on this thread (ADFFT_OK if none). */
int adfft_last_error(void);

/* Static, human-readable name of a status code. */
const char *adfft_status_string(int status);

/* Free the plan's device tables, workspace and graphs.  NULL is accepted.
 * Synchronises the device first so no launch of the plan is still running. */
int adfft_plan_destroy(adfft_plan_t plan);

/* Set the scale S (default 1/N, i.e. T/N with T = 1; S = T/N for a record of length T). */
int adfft_plan_set_scale(adfft_plan_t plan, double S);

/* Choose the algorithm; ADFFT_ERR_NOT_SUPPORTED if it cannot serve this plan's sizes. */
int adfft_plan_set_algorithm(adfft_plan_t plan, int algo);

/* Choose the FFT-stage arithmetic (adfft_precision_t); ADFFT_ERR_NOT_SUPPORTED if
 * the plan's dtype or algorithm has no such form. */
int adfft_plan_set_precision(adfft_plan_t plan, int mode);

/*
 * Output range.  For a real signal the spectrum is Hermitian, X_{M-m} = conj X_m
 * (the negative frequencies of Sec. 2, Eq. 2), so bins 0 .. M/2 determine all M.
 * ADFFT_OUTPUT_HALF makes adfft_execute write only those M/2 + 1 bins
 * (d_out [batch][M/2 + 1]), half the output bytes; adfft_execute_adjoint then
 * takes d_grad_out [batch][M/2 + 1] and returns the adjoint of that map (the
 * real part of S A^H applied to the gradient extended by zeros above M/2).
 * Served for real plans with even N and M in the single-pass fold form
 * (ADFFT_ERR_NOT_SUPPORTED otherwise, the plan unchanged); such a plan keeps
 * to that form (adfft_plan_set_algorithm accepts only ADFFT_ALGO_FOLD and AUTO).
 */
int adfft_plan_set_output(adfft_plan_t plan, int mode);

/* Fill *info; ADFFT_ERR_INVALID_ARG for NULL arguments. */
int adfft_plan_get_info(adfft_plan_t plan, adfft_plan_info_t *info);

/* Device workspace bytes the plan holds (0 for the fused single-pass form). */
size_t adfft_plan_workspace_bytes(adfft_plan_t plan);

/*
 * Forward transform of the whole batch: d_in [batch][N] (input dtype),
 * d_out [batch][M] complex.  Both device pointers, 16-byte aligned, not
 * overlapping.  Asynchronous on `stream`.
 */
int adfft_execute(adfft_plan_t plan, const void *d_in, void *d_out, void *stream);

/*
 * Adjoint (conjugate-transpose) transform, the backward pass of adfft_execute:
 *     d_grad_in[n] = S * sum_m exp(+2 pi i m n / M) * d_grad_out[m]
 * for complex plans, and its real part for real plans (the adjoint with
 * respect to the real inner product, which is what a gradient needs).  With
 * S = 1/(alpha N) this is the inverse transform in the second line of Eq. 7.
 * d_grad_out [batch][M] complex; d_grad_in [batch][N] of the input dtype.
 */
int adfft_execute_adjoint(adfft_plan_t plan, const void *d_grad_out, void *d_grad_in,
                          void *stream);

/*
 * Synchronise `stream`, then read and clear the plan's device status word
 * (a ragged plan: the status word of every shape class).
 * Returns ADFFT_OK, or ADFFT_ERR_TIMEOUT if a kernel of the plan gave up a
 * bounded device-side wait (for example on an asynchronous copy) since the
 * last call; the outputs of the launches concerned are then invalid.  Kernels
 * never trap or spin without limit: a wait that runs out sets this word and
 * the kernel returns.
 */
int adfft_plan_sync_status(adfft_plan_t plan, void *stream);

/*
 * End-to-end forward transform from HOST memory: copies h_in to the device,
 * runs adfft_execute, copies the spectrum back to h_out and synchronises the
 * stream.  The device staging buffers are allocated by the plan on first use
 * and kept until adfft_plan_destroy.  Host buffers should be page-locked for
 * full copy bandwidth.  Returns after the stream is synchronised, with the
 * plan's status word checked as by adfft_plan_sync_status.
 */
int adfft_execute_host(adfft_plan_t plan, const void *h_in, void *h_out, void *stream);

/*
 * Autotuner.  The default rule picks, for the fold form, the longest
 * power-of-two sub-FFT g' dividing gcd(M, N) (halved for real input) whose
 * P' = M/g' residues fit one cluster's shared memory, with a fold of at most
 * 16 blocks (the fold identity holds for every divisor of the gcd), the
 * smallest such cluster, input staging where it fits, and as many clusters as
 * can be resident at once, each looping over signals; the two-pass form only
 * where no single-pass shape fits.  Its split g = A*B: for FP32 plans whose pass 1
 * has a residue count that is a multiple of 4 above 4, the longest A with B >= 512
 * whose pass 1 fits 4 CTAs (the forward's pass 1 then spreads each column's residues
 * over independent CTAs of 4 residues); otherwise the longest A whose pass 1 fits
 * one CTA, else clusters of up to 4, then 8.
 *
 * adfft_plan_autotune times the forward transform of the plan (flags 0) or the
 * forward transform and its adjoint (ADFFT_TUNE_WITH_ADJOINT) for every
 * candidate launch shape (sub-FFT length, cluster size, input staging, a
 * resident-size or one-per-signal grid; the two-pass form, with every split
 * of its transform length into A*B, where it applies) with `iters` timed launches each (1..100;
 * 0 means 3) on the caller's buffers, times the candidates within 5 % of the
 * fastest (at most three) again in three alternating rounds, keeps the one with
 * the smallest time, and records it in
 * the process-wide tuning cache under (GPU name, driver version, N, M, batch,
 * dtype, precision).  d_in and d_out are as for adfft_execute (d_out is
 * overwritten); for a ragged plan the packed buffers, and every shape class
 * is tuned.  The call synchronises `stream` and must not run while the stream
 * is being captured.  Returns ADFFT_OK, or the first error of a launch.
 *
 * Plans created later with the same sizes on the same GPU model and driver
 * take the cached shape; entries of another GPU or driver are kept but never
 * used.  adfft_autotune_save writes the cache to a JSON file, and
 * adfft_autotune_load merges a file written by it (ADFFT_ERR_INVALID_ARG for
 * a file it cannot read or parse; nothing is merged then).
 * adfft_autotune_clear empties the cache.  The cache is guarded by a mutex;
 * a plan itself is not thread-safe.
 */
int adfft_plan_autotune(adfft_plan_t plan, const void *d_in, void *d_out, void *stream, int iters,
                        int flags);

/* Flags of adfft_plan_autotune: time each candidate on a forward transform followed by
 * its adjoint (the backward pass of a training step) instead of the forward alone.  The
 * adjoint writes into a temporary device buffer of the input's size that the call
 * allocates and frees.  The cache keeps one entry per key: the last tuning wins. */
#define ADFFT_TUNE_WITH_ADJOINT 1

/*
 * Set the fold form's launch shape by hand (the autotuner's candidates):
 * fft_len = the sub-FFT length g' (a power of two dividing M and N, halved for
 * real input; 0 = the largest such), cluster = CTAs per signal (0 = the
 * smallest that fits), staged = 1 to stage each signal through shared memory,
 * 0 not to, -1 where it fits, 2 for the push-exchange form (real fp32 input, one
 * residue per CTA, cluster = the number of residues: each CTA bulk-copies the runs
 * of its residue that the other CTAs need into their shared memory instead of the
 * CTAs loading them from one another; served for the compile-time shapes the
 * library instantiates, ADFFT_ERR_NOT_SUPPORTED otherwise); grid = clusters launched: 0 = as many as can be
 * resident at once, each looping over signals (the default), -1 = one per
 * signal, n > 0 = at most n.  Selects the fold algorithm.  Returns
 * ADFFT_ERR_NOT_SUPPORTED (the plan unchanged) when the shape does not fit
 * one cluster or the plan has no fold form (ragged, or chirp-z only sizes).
 */
int adfft_plan_set_launch_shape(adfft_plan_t plan, int64_t fft_len, int cluster, int staged, int grid);
int adfft_autotune_save(const char *path);
int adfft_autotune_load(const char *path);
int adfft_autotune_clear(void);

/*
 * Forward transform that allocates no device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc at the point where they need the transform:
 * code running while a CUDA graph is being captured (an allocation there
 * would be captured or rejected), code whose device memory is entirely
 * owned by another allocator or a fixed pool, and latency-critical loops
 * where an allocation could block.  Such callers cannot create a plan
 * (plan creation allocates tables and workspace), so this call takes the
 * sizes directly and returns when the work is queued on `stream`.
 *
 * Arguments: N samples and M = alpha*N bins per signal, `batch` signals,
 * dtype ADFFT_R32 or ADFFT_C64 (others: ADFFT_ERR_NOT_SUPPORTED); d_in
 * [batch][N] and d_out [batch][M] complex64 device buffers owned by the
 * caller, 16-byte aligned and not overlapping; scale S = 1/N.  The result
 * is the same transform as adfft_execute, computed with the two-pass
 * (four-step) form.
 *
 * Storage: the pass-1 intermediate and the twiddle tables live in one fixed
 * static device array of the library (1 MiB of tables + 32 MiB of scratch),
 * which every GPU that loads the library keeps until the process exits.
 * Limits: N/2 (real) or N (complex) a power of two >= 4, real input with
 * even N and M, batch * M/2 (real) or batch * M (complex) complex64 values
 * within the 32 MiB scratch, M < 2^30; larger requests return
 * ADFFT_ERR_UNSUPPORTED_SIZE without launching anything.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once for that device; make that first call before
 * any stream capture begins.  Every call reuses the same array and leaves the
 * last call's contents in it; nothing in it needs to start at zero.  The
 * tables are rewritten (four small kernels) only when a call's sizes differ
 * from those of the previous call on the same device.  Calls
 * whose work overlaps on the GPU (for example on two streams) race on the
 * array and produce wrong results: serialise them.
 */
int adfft_execute_noalloc(int64_t N, int64_t M, int64_t batch, int dtype, const void *d_in,
                          void *d_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ADFFT_H */
