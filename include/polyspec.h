/*
 * polyspec.h -- C ABI of the GB300 (sm_103a) unbiased polyspectrum estimator.
 *
 * The library estimates the power spectrum S2, the bispectrum S3 and the
 * two-dimensional trispectrum cut S4 of one or more real signal channels with
 * the unbiased multivariate k-statistics of arXiv 2505.01231 ("Correct
 * Estimation of Higher-Order Spectra ... in SignalSnap"):
 *
 *   frames ................ Sec. 3, Eq. 16: frame j of a channel is z[jT .. jT+T-1]
 *   window ................ Sec. 3, Eq. 17; App. B, Eq. 71 (confined Gaussian)
 *   Fourier coefficients .. Sec. 3, Eq. 18: X_k = sum_i g_i z_i exp(+2 pi j ik/T),
 *                           k = 0..T/2 (positive exponent, t0 = 0)
 *   k-statistics .......... Sec. 4.1, Eq. 32-34 over a group of m consecutive frames;
 *                           the fourth order in the factorised form of App. H, Eq. 85
 *   spectra ............... Sec. 3, Eq. 23 (S2); Sec. 4, Eq. 28 (S3), Eq. 31 (S4 cut);
 *                           Sec. 7, Eq. 47, 48, 50 (multi-channel)
 *   error bars ............ Sec. 4.2, Eq. 35-36 with the parts N_p = the groups
 *
 * Notation: T = samples per frame (the paper's N), dt = sample interval (the
 * paper's T/N), M = T/2 + 1 bins, m = frames per group, G = groups.  With
 * a_k = dt X_k the normalisations read
 *   S2 = dt c2(X_k, X_k*) / sum g^2,  S3 = dt^2 c3(X_k, X_l, X_{k+l}*) / sum g^3,
 *   S4 = dt^3 c4(X_k, X_k*, X_l, X_l*) / sum g^4.
 * Each group gives one estimate S_g; the result is the mean over groups and
 * the standard error sqrt(G/(G-1) (mean(x^2) - mean(x)^2) / G) of x = Re S_g and
 * of x = Im S_g separately.
 *
 * Conventions shared by every call:
 *  - No exception or abort crosses the ABI: every call returns an ss_status and
 *    ss_last_error() describes the last failure of a plan.
 *  - A plan owns all of its device memory (window, twiddles, carry-over samples,
 *    centred-spectrum scratch, FP64 accumulators).  The caller owns every input
 *    and output buffer it passes.
 *  - All device work of a plan is ordered on the stream given to ss_plan (NULL =
 *    the legacy default stream).  A plan must not be used by two host threads at
 *    the same time.
 *  - Pointers may be device pointers or host pointers (pinned or pageable); the
 *    library inspects each pointer with cudaPointerGetAttributes.
 */
#ifndef POLYSPEC_H
#define POLYSPEC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ss_plan_s* ss_plan_t;
typedef struct ss_many_s* ss_many_t;

typedef enum {
  SS_OK = 0,
  SS_EINVAL = -1,       /* an argument is out of range or inconsistent            */
  SS_ENOMEM = -2,       /* a device or pinned-host allocation failed               */
  SS_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed             */
  SS_ESTATE = -4,       /* the call is not valid in the plan's current state       */
  SS_ETIMEOUT = -5,     /* a bounded device-side wait gave up                      */
  SS_EUNSUPPORTED = -6  /* valid request that this build does not implement        */
} ss_status;

/* window kinds (Sec. 3, Eq. 17) */
enum { SS_WIN_HANN = 0, /* periodic Hann, g_i = 0.5 - 0.5 cos(2 pi i / T)            */
       SS_WIN_ACG = 1   /* approximate confined Gaussian, App. B, Eq. 71; win_param
                           is sigma_t (the paper's default is 0.14)                  */ };

/* spectral orders, OR-ed together; SS_ORDER1 is the first-order spectrum of
   each channel, S1 = N C1(a_0) / (T sum g) (Sec. 4, App. G), read with
   ss_finalize_s1 */
enum { SS_ORDER1 = 1u << 1, SS_ORDER2 = 1u << 2, SS_ORDER3 = 1u << 3, SS_ORDER4 = 1u << 4 };

/* cumulant estimators (ss_set_estimator): the unbiased k-statistics of Sec. 4.1
   (Eq. 32-34, the default), or the natural estimators the paper compares them
   with (Sec. 4.1, Fig. 6): the cumulants of each group's m samples taken as a
   distribution of their own, biased for finite m */
enum { SS_EST_UNBIASED = 0, SS_EST_NATURAL = 1 };

/* sample type of the input chunks */
enum { SS_F32 = 0, /* float32 samples                                          */
       SS_I16 = 1  /* int16 ADC samples, converted exactly to float32           */ };

/* arithmetic of the fourth-order moment sums (S4); the rest is always FP32
   with FP64 cross-group accumulation and an FP64 combine */
enum { SS_PREC_FP32 = 0,    /* FP32 FMA on CUDA cores                          */
       SS_PREC_TF32X3 = 1,  /* tensor cores, TF32 hi/lo split, 3 products      */
       SS_PREC_BF16X3 = 2,  /* tensor cores, BF16 hi/lo split, 3 products      */
       SS_PREC_BF16 = 3,    /* tensor cores, plain BF16 inputs                 */
       SS_PREC_FP16X3 = 4   /* tensor cores, FP16 hi/lo split of operands scaled
                               by a power of two per bin, 3 products           */ };
/* Accuracy: FP32, TF32X3 and FP16X3 carry every operand to about 2^-22 and meet
   1e-5 of each spectrum's peak against the FP64 definition in the tested shapes
   (at T = 8, m = 5 the S4 reached 1.4e-5 of its peak in FP32 and about 1e-4 in
   the split modes: the terms of Eq. 85 cancel strongly there); BF16X3 carries them
   to about 2^-17 (its tests hold it to 5e-5) and plain BF16 to 2^-9: both are
   outside that bar.  FP16X3 runs the products at the BF16 rate (twice TF32's)
   with TF32X3's accuracy: each bin's operands are multiplied by a power of two
   that keeps them inside the FP16 range, which the kernel divides out exactly. */
/* The tensor-core precisions contract the weighted frame Gram of each bin
   (m(m+1)/2 products per grid point and group) and take m <= 32 when a
   one-channel plan computes S4; ss_plan returns SS_EUNSUPPORTED for larger m.
   Plans of several channels compute every S4 combination C4(a_k, b_k*, c_l,
   d_l*) in FP32 on CUDA cores with SS_PREC_FP32, and on the tensor cores (five
   complex frame products per combination and group, Sec. 7, Eq. 50, App. H,
   Eq. 85; any m) in FP16X3 with SS_PREC_FP16X3 (each bin's operands scaled by a
   power of two per group) and in TF32X3 with the other tensor-core precisions,
   so their accuracy is that of FP16X3 or TF32X3.  All precisions
   keep the per-group c4 values and their per-item sums in FP32: inputs whose
   |c4| exceeds about 1e18 overflow the sum of squares. */

/* Size and layout information of a plan (filled by ss_query). */
typedef struct {
  int channels, T, M, m;
  int n_s2, n_s3, n_s4;      /* number of channel combinations per order          */
  int rows3, rows4;          /* rows of each S3 / S4 grid: M (one channel) or 2M-1 */
  long long groups;          /* groups accumulated since the last reset           */
  long long samples;         /* samples per channel consumed since the last reset */
  long long carried;         /* samples per channel waiting for a full group      */
  int groups_per_batch;      /* groups processed per device batch                 */
  size_t device_bytes;       /* device memory held by the plan                    */
  int kernels_per_batch;     /* kernel launches of one device batch (the K1-K3
                                stages of this window set; the interlaced set, if
                                any, launches as many again)                      */
} ss_info;

/* Per-stage device time, summed over launches since the last reset, measured
   with CUDA events on the plan's stream when timing is enabled
   (ss_set_timing).  Index 0: frame/window/FFT/centre + S2 (K1); 1: S3 (K2);
   2: S4 (K3); 3: finalize (K4); 4: host<->device copies. */
typedef struct {
  double ms[5];
  long long launches[5];
  long long pairs3;          /* bispectrum grid points evaluated per group        */
  long long pairs4;          /* trispectrum grid points evaluated per group       */
} ss_stats_t;

/*
 * ss_plan -- create a plan.
 *   out        receives the plan handle (set to NULL on failure).
 *   channels   number of real channels C, 1 <= C <= 4.
 *   T          samples per frame, a power of two in [8, 4096] (Eq. 16-18).
 *   dt         sample interval, > 0 (the paper's T/N).
 *   m          frames per group (k-statistic sample size, Sec. 4.1); m >= 2 for
 *              S2, m >= 3 with SS_ORDER3, m >= 4 with SS_ORDER4 (the c3 and c4
 *              prefactors of Eq. 33-34 divide by m-2 and m-3).
 *   window     SS_WIN_HANN or SS_WIN_ACG; win_param = sigma_t for SS_WIN_ACG.
 *   orders     OR of SS_ORDER1/2/3/4, at least one.
 *   dtype      SS_F32 or SS_I16.
 *   precision  SS_PREC_* for the S4 moment sums.
 *   combos     NULL for the default combinations, else n_combos records of five
 *              ints {order, c0, c1, c2, c3} (channels c0.. of the cumulant of
 *              Eq. 47 (order 2: C2(c0_k, c1_k*)), Eq. 48 (order 3:
 *              C3(c0_k, c1_l, c2_{k+l}*)) or Eq. 50 (order 4:
 *              C4(c0_k, c1_k*, c2_l, c3_l*)); unused entries are ignored.
 *              Defaults: one channel -> the auto spectra of each requested
 *              order; several channels -> every multiset of channels for S2 and
 *              S3 and every distinct pairing for S4 (ss_query gives the counts;
 *              ss_combos lists them).
 *   stream     cudaStream_t on which all device work is ordered (NULL = default).
 * Errors: SS_EINVAL for out-of-range arguments, SS_ENOMEM, SS_ECUDA,
 * SS_EUNSUPPORTED for combinations this build does not implement.
 */
ss_status ss_plan(ss_plan_t* out, int channels, int T, double dt, int m, int window,
                  double win_param, unsigned orders, int dtype, int precision,
                  const int* combos, int n_combos, void* stream);

/*
 * ss_accumulate -- feed the next n_samples samples of every channel.
 *   chunk      [channels][n_samples] samples of the plan's dtype, channel-major
 *              (channel c starts at element c * n_samples).  Device memory or
 *              host memory (pinned or pageable).
 * The record is cut into consecutive frames of T samples and groups of m frames
 * (Eq. 16; Sec. 10 estimates from m consecutive windows).  Samples that do not yet
 * complete a group are kept by the plan and prepended to the next chunk, so any
 * split of a record into chunks gives the same groups and the same result.
 * Work is enqueued on the plan's stream; a device chunk must stay valid until
 * that stream has passed the call, a host chunk may be reused when the call
 * returns.
 * Errors: SS_EINVAL (NULL chunk with n_samples > 0), SS_ESTATE (after a failed
 * launch), SS_ECUDA.
 */
ss_status ss_accumulate(ss_plan_t plan, const void* chunk, size_t n_samples);

/*
 * ss_finalize -- write the spectra accumulated since the last reset.
 * Outputs are complex128 values stored as interleaved (re, im) doubles; each
 * error array holds (err_re, err_im) pairs in the same layout.  Any pointer may
 * be NULL to skip that output; any may be host or device memory.
 *   S2   [n_s2][M]
 *   S3   [n_s3][rows3][M]; one channel: rows3 = M, element (k, l) for k, l >= 0,
 *        zero outside k + l <= M-1.  Several channels: rows3 = 2M-1, row r holds
 *        k = r - (M-1), zero outside |k + l| <= M-1.
 *   S4   [n_s4][rows4][M]; one channel: rows4 = M, (k, l) for k, l >= 0.
 *        Several channels: rows4 = 2M-1, row r holds k = r - (M-1).
 * The plan keeps its sums: more ss_accumulate calls may follow.
 * Leftover samples that never completed a group do not enter the result.
 * Errors: SS_ESTATE if fewer than two groups were accumulated (no error bar,
 * Eq. 35 divides by N_p - 1), SS_ECUDA.  Synchronises the plan's stream.
 */
ss_status ss_finalize(ss_plan_t plan, double* S2, double* S3, double* S4,
                      double* S2_err, double* S3_err, double* S4_err);

/*
 * ss_finalize_s1 -- first-order spectrum of every channel (a plan made with
 *   SS_ORDER1): S1 [channels] complex128 interleaved (re, im) and S1_err
 *   [channels][2] (standard errors of Re and Im over the groups, Eq. 35-36),
 *   host or device memory; either may be NULL.  S1 is the group-averaged mean
 *   of the zero-frequency coefficient divided by sum g, i.e. the window-
 *   weighted mean of the signal.  SS_ESTATE with fewer than two groups or
 *   without SS_ORDER1.  Synchronises the plan's stream.
 */
ss_status ss_finalize_s1(ss_plan_t plan, double* S1, double* S1_err);

/*
 * ss_set_estimator -- SS_EST_UNBIASED (default) or SS_EST_NATURAL for every
 *   order of the plan.  Valid only before the first ss_accumulate (or after
 *   ss_reset); SS_ESTATE otherwise, SS_EINVAL for another value.
 */
ss_status ss_set_estimator(ss_plan_t plan, int estimator);

/*
 * ss_set_interlace -- on (1) or off (0): interlaced spectra (Sec. 3).  The plan
 *   also frames the record from its sample T/2 on (windows shifted by half a
 *   frame, so the middle of one window set covers the edges of the other) and
 *   pools the groups of both window sets in every estimate and error bar; with
 *   as many groups in each set, the estimate is the average of the two spectra.
 *   The error bar (Eq. 35-36) treats all pooled groups as independent parts,
 *   which the overlapping windows of the two sets are not quite: it is somewhat
 *   optimistic.
 *   Doubles the work and the device memory.  Valid only before the first
 *   ss_accumulate (or after ss_reset); SS_ESTATE otherwise.  ss_query reports
 *   the pooled groups; ss_export_state writes the pooled sums.
 */
ss_status ss_set_interlace(ss_plan_t plan, int on);

/*
 * Sequential spectra (Sec. 8, quasi-polyspectra of non-stationary signals):
 * besides the whole-record estimate, the short-time estimates of the record,
 * averaged over blocks of consecutive groups.
 *
 * ss_set_sequential -- every block_groups consecutive groups (counted from the
 *     first group after ss_plan or ss_reset, across ss_accumulate calls), the
 *     plan writes the block's S2, S3 and S4 -- the mean of the block's
 *     per-group estimates S_g and its standard error over those groups
 *     (Eq. 35-36 with the block's groups as the parts), i.e. the estimate of
 *     that stretch of the record -- to block b of out: ss_sequential_info gives
 *     the doubles per block, laid out as the six outputs of ss_finalize in the
 *     order S2, S2_err, S3, S3_err, S4, S4_err.  Blocks b >= max_blocks are
 *     counted but not written.  out is device memory (SS_EINVAL otherwise); it
 *     may be NULL with max_blocks = 0.  block_groups = 0 turns the blocks off;
 *     1 is SS_EINVAL (a block needs two groups for its error bar).  Valid only
 *     before the first ss_accumulate (or after ss_reset); SS_EUNSUPPORTED with
 *     interlaced window sets.  Groups after the last whole block enter the
 *     whole-record estimate only.  Stream-ordered: a block is written when the
 *     plan's stream passes the ss_accumulate call that completed it.
 * ss_sequential_info -- the doubles of one block, and the blocks completed since
 *     the last reset (either pointer may be NULL).
 * A sweep of m (Sec. 8: quasi-polyspectra that change with m reveal
 * non-stationarity) is a plan per m over the same record.
 */
ss_status ss_set_sequential(ss_plan_t plan, int block_groups, double* out, long long max_blocks);
ss_status ss_sequential_info(ss_plan_t plan, size_t* block_doubles, long long* blocks_done);

/*
 * Complex-valued signals (App. D) and S4 planes off the cut (App. E).
 *
 * A complex signal z = x + j y is fed as its two real channels (x and y among
 * the plan's channels), so any mix of real and complex signals fits in one
 * plan.  An operand is three ints {re, im, conj}: the real channel carrying the
 * real part, the one carrying the imaginary part (-1 for a real signal), and 1
 * for the conjugate signal z* (else 0).  With A, B, C, D the Fourier
 * coefficients of the operands (Eq. 18, positive exponent) at signed bins, and
 * the window and dt normalisation of Eq. 23, 28, 31:
 *   order 2: S2(k)    ~ c2(A(k), B(-k))                        [2M-1]
 *   order 3: S3(k, l) ~ c3(A(k), B(l), C(-k-l))                [2M-1][2M-1]
 *   order 4: S4(k, l) ~ c4(A(k+s), B(-k-s), C(l-s), D(-l+s))   [2M-1][2M-1]
 * with k = row - (M-1), l = column - (M-1), bins mod T, S3 zero where
 * |k + l| > M-1.  For real operands these are the spectra of Eq. 47, 48, 50 on
 * the whole plane; for complex ones they are the multilinear combinations that
 * App. D writes as sums of 4, 8 or 16 real spectra, taken per group, so the
 * error bars (Eq. 35-36) are those of the combination.  s = s4_shift moves the
 * S4 plane through the 3-D trispectrum: it is the cut of the signals
 * z1 e^{j dw t}, z2 e^{-j dw t}, z3 e^{-j dw t}, z4 e^{j dw t}, dw = 2 pi s/(T dt).
 *
 * ss_set_complex      -- n records of 13 ints {order, op0 (3 ints), op1, op2,
 *     op3} (unused operands ignored) and the shift; replaces any earlier set.
 *     Valid only before the first ss_accumulate (or after ss_reset).
 *     SS_EINVAL for a bad order, channel or flag; SS_EUNSUPPORTED with
 *     interlaced window sets.  The sums are not part of exported states.
 * ss_complex_size     -- doubles of the means of all records (the same again
 *     for the errors): per record 2 (2M-1) (order 2) or 2 (2M-1)^2.
 * ss_finalize_complex -- the records' means (complex128 interleaved) and errors
 *     ((err_re, err_im) pairs), concatenated in record order; host or device
 *     memory, either may be NULL.  Synchronises the plan's stream.
 */
ss_status ss_set_complex(ss_plan_t plan, const int* records, int n_records, int s4_shift);
ss_status ss_complex_size(ss_plan_t plan, size_t* n_doubles);
ss_status ss_finalize_complex(ss_plan_t plan, double* S, double* S_err);

/*
 * ss_inject_timeout -- fault-injection hook for testing the timeout path (no
 *   counterpart in the paper).  Every kernel that waits for its own staged data
 *   (TMA copies, tensor-core products) bounds each wait by 2 s of %globaltimer;
 *   a wait that runs out records SS_ETIMEOUT in the plan's device status word,
 *   and its CTA waits (with the full limit) for the copies it has issued, frees
 *   its tensor memory and returns, so the device stays usable.  The next
 *   ss_finalize, ss_finalize_s1 or ss_export_state then returns SS_ETIMEOUT and
 *   the plan is unusable (SS_ESTATE) from then on.  With on = 1, every
 *   bispectrum launch of the plan (orders with SS_ORDER3) makes one such wait
 *   run out: at the first step of its first work item, after that step's copies
 *   are issued, one thread waits 1 ms on a barrier that nothing completes.  On
 *   = 0 turns it off.  Nothing faults, traps or hangs.
 */
ss_status ss_inject_timeout(ss_plan_t plan, int on);

/*
 * Autotuning of the kernel forms (Sec. 10 names autotuning in the style of
 * FFTW as a direction for the library; the paper gives no procedure).  A plan's
 * results do not depend on these choices, only its speed: K1 keeps a group's
 * coefficients in shared memory within a 74 KB or a 96 KB budget, or with a
 * warp per frame (T <= 1024), or transforms one frame at a time; K2 uses 4 x 4
 * micro-tiles in CTAs of 256 threads (4 stages, or 3 stages with three CTAs per
 * SM), 8 x 4 micro-tiles in CTAs of 128 threads with 2 or 3 pipeline stages, or
 * (one channel) 8 x 4 micro-tiles in warps that each take their own 32 x 32
 * sub-tiles and stage their own frames, with no block barrier.
 *
 * ss_autotune   -- time every form of K1 and K2 on this plan's shapes on this
 *                  GPU (a synthetic Gaussian record of about 64 x SMs groups,
 *                  generated on the device; one untimed pass and the best of
 *                  three per form) and keep the fastest.  Valid only before the
 *                  first ss_accumulate (or after ss_reset); SS_ESTATE otherwise.
 *                  Allocates and frees that record; synchronises the plan's
 *                  stream; leaves the plan reset.  best_ms (may be NULL)
 *                  receives the time of the fastest pass.
 * ss_get_tuning -- the plan's choices as text: "polyspec-tuning 1 <key> |
 *                  k1=<auto|r96|frames|warp> k2=<44|44s3|84s2|84s3|84w>", where the key names
 *                  T, m, channels, dtype, precision, SM count and GPU.  out holds
 *                  cap bytes (SS_EINVAL if too small).
 * ss_set_tuning -- apply such a text (valid at any time between calls).  A text
 *                  with a key applies only to a plan of the same key (SS_EINVAL
 *                  otherwise); "k1=... k2=..." alone applies to any plan.
 */
ss_status ss_autotune(ss_plan_t plan, double* best_ms);
ss_status ss_get_tuning(ss_plan_t plan, char* out, size_t cap);
ss_status ss_set_tuning(ss_plan_t plan, const char* text);

/* ss_reset -- zero the accumulators, the carry-over and the statistics. */
ss_status ss_reset(ss_plan_t plan);

/* ss_query -- sizes and layout of the plan's outputs (see ss_info). */
ss_status ss_query(ss_plan_t plan, ss_info* info);

/* ss_layout -- the work decomposition that a plan of this shape uses, computed
   on the host (no device call, no plan).  S3 (Eq. 28 / Eq. 48 domain): the
   64 x 64 tiles of (k, l) that K2 takes, as (k0, l0) pairs in s3_tiles, and the
   grid points left to the point kernel (tiles holding at most 8 domain points,
   one channel only), as (k, l) pairs in s3_points.  S4 on tensor cores (one
   channel): the tiles of the upper triangle k <= l as (k0, l0, columns) triples
   in s4_tiles, and last_col = 1 when the column l = M - 1 is left to the
   CUDA-core column kernel.  Each array receives at most its max entries (it may
   be NULL); n3, np and n4 receive the full counts.  Errors: SS_EINVAL for
   channels outside [1, 4], T not a power of two in [8, 4096], or a NULL count. */
ss_status ss_layout(int channels, int T, int* s3_tiles, int max3, int* n3, int* s3_points,
                    int maxp, int* np, int* s4_tiles, int max4, int* n4, int* last_col);

/* ss_layout_warps -- the S3 decomposition of the independent-warp K2 form (one
   channel; host only, no device call): the 32 x 32 sub-tiles of (k, l) that hold
   more than 8 points of the domain 0 <= k <= l, k + l <= M - 1 (Eq. 28), as
   (k0, l0) pairs in tiles, and the domain points of the other sub-tiles, left to
   the point kernel, as (k, l) pairs in points.  Each array receives at most its
   max entries (it may be NULL); n and np receive the full counts.  Errors:
   SS_EINVAL for T not a power of two in [8, 4096], or a NULL count. */
ss_status ss_layout_warps(int T, int* tiles, int max_tiles, int* n, int* points, int maxp,
                          int* np);

/* ss_combos -- copy the plan's combinations, (n_s2 + n_s3 + n_s4) records of
   five ints {order, c0, c1, c2, c3} in output order; out may hold max_records. */
ss_status ss_combos(ss_plan_t plan, int* out, int max_records);

/* ss_set_timing -- enable (1) or disable (0) per-stage CUDA-event timing. */
ss_status ss_set_timing(ss_plan_t plan, int enable);

/* ss_stats -- per-stage device times (synchronises the plan's stream). */
ss_status ss_stats(ss_plan_t plan, ss_stats_t* stats);

/* ss_set_batch -- cap on groups per device batch (0 = automatic).  Changing it
   only changes scheduling, never the result.  Valid only right after ss_plan or
   ss_reset. */
ss_status ss_set_batch(ss_plan_t plan, int groups_per_batch);

/*
 * Sharding a record across GPUs or processes (Sec. 4.2: the estimate and its
 * error bar of Eq. 35-36 are built from sums over groups of the per-group
 * spectra S_g and of (Re S_g)^2, (Im S_g)^2, so plans that saw disjoint sets of
 * whole groups combine by adding those sums).
 *
 * A state is SS_STATE_HEADER doubles followed by the plan's float64 sums.
 * Header words 0..13 describe the configuration (channels, T, m, orders,
 * precision, window, sigma_t, dt, the number of S2/S3/S4 combinations, a
 * 52-bit hash of the combination list, a layout version, the estimator) and
 * must match between plans that are merged; word 14 is the number of groups,
 * word 15 the number of samples per channel in them.
 * Samples carried over towards an incomplete group are not part of a state.
 *
 * ss_state_size   -- number of doubles of the plan's state (header included).
 * ss_export_state -- write the state to dst (host or device memory, at least
 *                    ss_state_size doubles).  Synchronises the plan's stream.
 * ss_merge_state  -- add a state written by ss_export_state of a plan with the
 *                    same configuration (host or device memory): its group
 *                    sums, groups and samples are added to this plan's.  A
 *                    configuration mismatch returns SS_EINVAL and changes
 *                    nothing.  Stream-ordered; a host src is copied before the
 *                    call returns.
 * Adding exported states element-wise (e.g. an all-reduce sum) and merging
 * the total into a reset plan gives the state of the union of the groups.
 */
#define SS_STATE_HEADER 16
ss_status ss_state_size(ss_plan_t plan, size_t* n_doubles);
ss_status ss_export_state(ss_plan_t plan, double* dst);
ss_status ss_merge_state(ss_plan_t plan, const double* src);

/*
 * Many independent recordings in one CUDA graph (Sec. 3, Eq. 16-18 per
 * recording; the estimate of each recording is the same as a one-channel
 * ss_plan's).  Each recording has its own frame length and length and gets
 * its own S2, S3 and S4 with error bars.
 *
 * ss_plan_many -- one-channel plans for n_rec recordings: T[i] is recording
 *     i's frame length (a power of two in [8, 4096]), max_samples[i] the most
 *     samples it will be given (at least two groups, m T[i] each); dt, m,
 *     window, win_param, orders and precision are shared and mean what they
 *     mean for ss_plan; stream is the cudaStream_t the runs are ordered on.
 *     The device scratch of all recordings together is about 6 GiB; longer
 *     recordings are processed in several batches inside the graph.
 * ss_run_many -- for every recording i: reset, accumulate the n_samples[i]
 *     float32 samples at chunks[i] (device memory) and finalize into S2[i],
 *     S3[i], S4[i] and the *_err[i] (layouts as for ss_finalize of a
 *     one-channel plan; device or page-locked host memory; a NULL list or
 *     entry skips that output).  The first call captures all of it as one CUDA
 *     graph (the recordings one after the other on one stream, longest first)
 *     and launches it; later calls with the same chunks, n_samples and outputs
 *     replay the graph, other arguments capture a new one.  ss_plan_many runs
 *     ss_autotune on one plan of each frame length and gives its choice to the
 *     other plans of that length (ss_get_tuning on ss_many_plan shows it).
 *     Synchronises the
 *     stream; returns SS_ETIMEOUT if a device-side wait of any recording gave
 *     up.  The arrays are host arrays of n_rec entries.
 * ss_many_plan -- the plan of recording i (owned by the handle; ss_query,
 *     ss_stats, ss_export_state work on it; do not destroy it).
 * ss_destroy_many -- release everything (NULL is accepted).
 * ss_many_last_error -- text of the handle's last failure (or of the last
 *     failed ss_plan_many when NULL).
 */
ss_status ss_plan_many(ss_many_t* out, int n_rec, const int* T, const size_t* max_samples,
                       double dt, int m, int window, double win_param, unsigned orders,
                       int precision, void* stream);
ss_status ss_run_many(ss_many_t many, const void* const* chunks, const size_t* n_samples,
                      double* const* S2, double* const* S3, double* const* S4,
                      double* const* S2_err, double* const* S3_err, double* const* S4_err);
ss_status ss_many_plan(ss_many_t many, int i, ss_plan_t* plan);
ss_status ss_destroy_many(ss_many_t many);
const char* ss_many_last_error(ss_many_t many);

/* ss_destroy -- release every resource of the plan (NULL is accepted). */
ss_status ss_destroy(ss_plan_t plan);

/* ss_last_error -- text of the last failure of the plan, or of the last failed
   ss_plan when plan is NULL.  Valid until the next call on the same plan. */
const char* ss_last_error(ss_plan_t plan);

/* ss_version -- library version string. */
const char* ss_version(void);

/*
 * ss_s2_noalloc -- power spectrum S2 of one float32 channel, without allocating
 * any device memory.  The paper has no counterpart to this entry point; it
 * exists for callers that cannot call cudaMalloc: processes whose device memory
 * is owned up front by a framework's caching allocator or by a fixed budget,
 * and latency-critical loops that must neither wait for an allocation
 * (cudaMalloc can synchronise the device) nor handle its failure.
 *
 * It computes the same S2, with the same error bars, as a one-channel plan with
 * SS_ORDER2 fed the whole record in one ss_accumulate call, with every
 * intermediate (window and twiddle tables, built on the device; centred
 * spectra; float64 sums) kept in one static device array of
 * SS_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library holds
 * until the process exits.  The call enqueues kernels and memsets only.
 *   d_signal   device pointer to n_samples float32 samples.
 *   T, dt, m, window, win_param   as for ss_plan (m >= 2).
 *   d_S2       device output, [M] complex128 as interleaved (re, im) doubles.
 *   d_S2_err   device output [M] (err_re, err_im), or NULL.
 *   stream     cudaStream_t; the work is enqueued on it and the call returns
 *              without waiting (outputs are ready when the stream passes it).
 * Limit: the centred spectra of all groups must fit the scratch array,
 * floor(n_samples / (m T)) * m * (M rounded up to a multiple of 4) * 8 bytes
 * <= SS_NOALLOC_SCRATCH_BYTES - 128 KiB; longer inputs return SS_EINVAL.
 * Fewer than two groups return SS_ESTATE.  d_signal, d_S2 and d_S2_err must be
 * device (or managed) memory: any other pointer returns SS_EINVAL before
 * anything is enqueued.  ss_noalloc_last_error() describes
 * the last failure of the calling thread.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current); make that first call before
 * any stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (concurrent streams, or several host threads) race on it
 * and give wrong results; order them on one stream or serialise them.
 */
#define SS_NOALLOC_SCRATCH_BYTES (32u << 20)
ss_status ss_s2_noalloc(const float* d_signal, size_t n_samples, int T, double dt, int m,
                        int window, double win_param, double* d_S2, double* d_S2_err,
                        void* stream);
const char* ss_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* POLYSPEC_H */
