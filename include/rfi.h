/*
 * rfi.h -- C ABI of the B300 (sm_103a) online RFI flagging library.
 *
 * The library implements the online interference mitigation of Yatawatta, Boonstra
 * and Broekema, "Energy and polarization based online interference mitigation in
 * radio interferometry" (arXiv 2412.14775):
 *   - complex Stokes I, Q, U, V of every sample (Section 2, Eq. IQUV);
 *   - over each window of M consecutive samples, the spectral-kurtosis statistic
 *       tau = (M d + 1)/(M - 1) * (M S2 / (S1^2 + eps) - 1),
 *       S1 = sum |I|, S2 = sum |I|^2                    (Section 2.1, Table 1);
 *   - the directional statistic of the normalised polarisation vector, separately
 *     for the real and the imaginary parts of (Q, U, V):
 *       p = sqrt(q^2 + u^2 + v^2) + eps, r = |sum (q, u, v)/p| / M
 *                                                       (Section 2.2, Table 2);
 *   - window flag = (tau < s_low) OR (tau > s_high) OR (r_Re > gamma) OR
 *     (r_Im > gamma); a NaN statistic also flags       (Sections 2.1, 2.2);
 *   - flagged samples are left out of the time average and the weight of each
 *     averaged output is the unflagged fraction        (end of Section 2.1).
 *
 * Terms.  A "stream" is one subband: R = B * C rows, B = N(N+1)/2 baselines of N
 * stations including autocorrelations (Section 2: each of the N(N+1)/2 correlator
 * streams is mitigated separately) and C channels.  Each row is one (baseline,
 * channel) time series; rows are independent.  Blocks of T samples of all rows
 * arrive one after another; windows and averaging bins are counted from the
 * stream's first sample and continue across blocks.
 *
 * Conventions for every function:
 *   - Every function returns an rfi_status (int).  No C++ exception crosses the ABI.
 *   - Buffers passed to rfi_process_* are caller-owned DEVICE pointers (e.g. the
 *     data pointer of a CUDA tensor) unless the function name ends in _host.  The
 *     library checks that each is device-accessible and suitably aligned and returns
 *     RFI_EINVAL otherwise; it never dereferences a host pointer on the device.
 *   - A context owns its device state (averaging carry, task counter), allocated in
 *     rfi_create*; rfi_process_block and rfi_process_batch allocate nothing, do not
 *     synchronise the stream and may be captured in a CUDA graph.
 *   - One context is used by one host thread at a time; work for one context must
 *     be issued in stream order (a context's carry is read and written by each call).
 *   - A CUDA error seen by a context makes it sticky-failed (RFI_ESTATE) until
 *     rfi_reset.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the legacy
 *     default stream).
 */
#ifndef RFI_H
#define RFI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rfi_ctx rfi_ctx;

/* Input sample formats.  One sample = the 4 correlations xx, xy, yx, yy of one
 * (baseline, channel, time) point (Section 2, Eq. V), each as (re, im). */
typedef enum {
    RFI_C64  = 0,   /* float32 re, im x 4 = 32 bytes per sample                   */
    RFI_C32H = 1    /* IEEE binary16 re, im x 4 = 16 bytes per sample; arithmetic
                       after exact widening to float32 (FP16 storage, FP32 math)   */
} rfi_dtype;

/* Thresholds (Sections 2.1-2.3).  d: SK shape parameter; [s_low, s_high]: SK
 * acceptance interval; gamma: directional-statistic threshold; eps: the additive
 * constant of Tables 1 and 2 (added to S1^2 and to p).  Stored on the device as
 * float32 (the kernels compare in float32).  No value may be NaN, d must be finite,
 * eps finite and >= 0 and s_low <= s_high (else RFI_EINVAL).  Infinite bounds are
 * allowed and switch a test off: s_low = -inf and s_high = +inf never flag by SK, and
 * gamma >= 1 (r never exceeds 1) or +inf never by DS; gamma < 0 flags every window. */
typedef struct {
    double d, s_low, s_high, gamma, eps;
} rfi_thresholds;

typedef enum {
    RFI_OK           = 0,
    RFI_EINVAL       = 1,   /* bad argument: size, alignment, pointer kind, layout */
    RFI_ENOMEM       = 2,   /* device or pinned-host allocation failed in create   */
    RFI_ECUDA        = 3,   /* a CUDA runtime call failed (context becomes sticky) */
    RFI_ETIMEOUT     = 4,   /* a bounded device wait gave up (reserved)            */
    RFI_ESTATE       = 5,   /* context is sticky-failed, destroyed or misused      */
    RFI_EUNSUPPORTED = 6    /* valid request this build has no kernel for          */
} rfi_status;

/* Launch shape of the flagging kernel.  Zero fields mean "choose automatically".
 *   lanes_per_row  P: lanes of a warp that share one row; a power of two in
 *                  {1, 2, 4, 8, 16, 32}; each lane owns every P-th load unit of a
 *                  window (a load unit is 32 bytes: one C64 sample or two C32H
 *                  samples; 16 bytes = one sample for C32H when M is odd).
 *   warps_per_block  1..32.
 *   host_max_T     > 0: also allocate device staging for rfi_process_block_host
 *                  with blocks of up to host_max_T samples.
 *   host_chunks    row chunks pipelined by rfi_process_block_host (copy in,
 *                  compute and copy out overlap across chunks); 0 = 4.
 *   compensated    Kahan-compensated S1 and S2 (the SK moments): 1 = on, -1 = off,
 *                  0 = on for windows of M >= 64 samples.
 *   prefetch_bytes   size of one L2 prefetch group per row (128-byte lines split over
 *                  the row's lanes), rounded down to whole
 *                  windows (at least one); a multiple of 16; 0 = 1024.
 *   prefetch_groups  how many such groups each row keeps requested ahead of the
 *                  window being loaded; 0 or -1 = no prefetch (default).
 *   max_registers  register budget per thread of the single-stream kernel: 0 or 128
 *                  (default), 96 (20 resident warps per SM, two chunks of at most 2
 *                  load units in flight per lane; at most 4 warps per block), 80 or
 *                  64 (one chunk in flight, more resident warps; at most 8 warps per
 *                  block); below 128: lanes_per_row <= 8.  Results do not depend on it.
 *   window_F       channels per window footprint (0 = 1): a window is M consecutive
 *                  samples of F adjacent channels of one baseline, W = M F samples
 *                  (the time-frequency windows of Sections 3.2 and 4).  A power of two
 *                  dividing `channels`, with lanes_per_row * window_F <= 32.  The
 *                  statistics then have shape [3][B][C/F][T/M]; every channel of a
 *                  flagged footprint is flagged; averages stay per channel.
 *   precision      0 = float32 arithmetic (default).  1 = the mixed precision the
 *                  paper's reinforcement-learning agent chose (Tables 3 and 4): SK
 *                  groups 5 and 7 and DS groups 4-7 in IEEE binary16, the rest in
 *                  binary32, every operation rounded in the tables' order, eps =
 *                  2^-10 inside binary16 groups; one lane per row, time-only windows,
 *                  no Kahan.  Statistics are then binary16 values.
 *                  2 = binary16 arithmetic for binary16 input (RFI_C32H): the Stokes
 *                  parameters are formed in binary16 (half2 adds, round to nearest even);
 *                  every later product multiplies two binary16 values (exact in
 *                  float32) and every sum is float32 (S1, S2 with Kahan as usual, the
 *                  polarisation-vector sums, the averaging sums); the polarisation
 *                  vector is normalised by 1/sqrt(q^2 + u^2 + v^2 + eps^2).  Each Stokes
 *                  component carries one binary16 rounding (relative 2^-11), which
 *                  bounds the statistics' error (|d tau| <~ 4 2^-11 (|tau| + (Md+1)/
 *                  (M-1)), |d r| <~ 2 2^-11) and that of the averages (2^-11 of the
 *                  magnitudes averaged).  Direct loader, 128-register budget, plain
 *                  stores, no prefetch, partial windows or adaptive thresholds; any
 *                  lanes_per_row, lane_split and window_F.
 *   loader         0 = direct 32-byte global loads (default).  1 = the rows are
 *                  staged in shared memory a few windows at a time by cp.async.bulk
 *                  (TMA) copies, one per row and stage issued by the row's first lane,
 *                  that complete on one mbarrier per stage; the row's lanes then read
 *                  the same units as the direct loader.  Rows are padded so that the
 *                  reads spread over all banks.  Every stage wait is bounded (about
 *                  2 s); a wait that gives up sets the context's error word, read by
 *                  rfi_check.  Needs float32 arithmetic and lanes_per_row <= 8 (all
 *                  register budgets; Kahan with 128); results equal the direct loader's
 *                  with the same lanes_per_row.  Single-stream calls only: batches run
 *                  the direct loader (bit-identical results).  2 = the same staging
 *                  with one TMA tensor-tile copy (cp.async.bulk.tensor.2d) per warp
 *                  and stage instead of one copy per row: the block's rows as a 2-D
 *                  tensor map of 8-byte elements (encoded per launch), a tile of the
 *                  warp's rows x the padded row pitch (the extra bytes are the next
 *                  samples, or zeros past the row; rows past the last read as zeros).
 *                  lanes_per_row <= 4 (a tile's 128-byte aligned destination), at
 *                  most 2048 bytes of a row per stage, no Kahan; the same results.
 *   tma_stage_windows  windows of every row per stage (0 = 1).
 *   tma_stages     stages in flight per warp (0 = 2); shared memory per block must
 *                  stay within 227 KB.
 *   debug_inject_wait_timeout  1 = for testing failure detection only: the staged
 *                  loader expects 16 more bytes per stage than it copies, so every
 *                  stage wait gives up after about 1 ms and the error word is set.
 *   buffered_stores  1 = each row keeps the statistics of 4 windows and 4 flag words
 *                  in registers and writes them with one 16-byte store each (fewer
 *                  store instructions for small windows).  Taken where T/M is a
 *                  multiple of 4, the flag words of a row are too (M dividing 32) and
 *                  the buffers are 16-byte aligned, else the plain stores run.  Needs
 *                  the direct loader, float32 arithmetic, the 128-register budget, no
 *                  Kahan, lanes_per_row <= 4 and 1, 2 or 4 load units per chunk.
 *                  Results are identical.
 *   partial_windows  1 = blocks of any length T (even T for binary16 input with even
 *                  M): a window that a block leaves open is completed by the next
 *                  block(s).  Its raw samples wait in a device buffer of the context
 *                  (R M samples, allocated here), and its flags, statistics and the
 *                  averages it completes are returned by the call that completes it,
 *                  so a call's outputs cover the windows it completes (rfi_windows_for)
 *                  and may start up to M-1 samples before its block.  Results are bit
 *                  identical to any other split of the stream, including one block.
 *                  Needs the direct loader, float32 arithmetic, the 128-register
 *                  budget and plain stores (kernel instances of their own, so the
 *                  others carry no cost).  0 = T must be a multiple of M (default).
 *   adaptive       1 = online per-stream SK thresholds (the paper's Sec. 5 names online
 *                  threshold adaptation as future work; this is the build's form of
 *                  it): every footprint row keeps, on the device, a running estimate
 *                  of the mean and second moment of tau over its unflagged windows
 *                  (the n-th such window weighted max(alpha, 1/n)); once n >= n_warm
 *                  the row's SK test uses [mean - k_sigma sd, mean + k_sigma sd]
 *                  instead of [s_low, s_high].  A launch uses the thresholds of the
 *                  state at its start and advances the state window by window.  gamma
 *                  stays fixed.  Parameters: rfi_set_adaptation (defaults alpha =
 *                  1/64, k_sigma = 3, n_warm = 32).  Needs the direct loader, float32
 *                  arithmetic, the 128-register budget, plain stores and whole
 *                  windows.
 *   overlap_bytes  launch overlap of consecutive single-stream calls (programmatic
 *                  dependent launch).  The flagging kernel is launched so that its
 *                  blocks may start while the kernel before it on the stream is still
 *                  finishing; until that kernel has completed they only request the
 *                  first overlap_bytes of their rows into L2 (a hint, safe whatever
 *                  that kernel writes), then wait for it and run as usual.  Results are
 *                  identical; back-to-back calls lose less time at each launch
 *                  boundary.  0 = 512 bytes (default), -1 = off, else a multiple of
 *                  128.  Launches recorded into a CUDA graph, the shared-memory loader
 *                  and batches keep plain stream order.  The library orders every
 *                  flagging launch against the flagging launches (of any context, and
 *                  of rfi_process_block_noalloc) that may still run on the same stream:
 *                  it waits as described only while each of those waited for the one
 *                  before it, and is otherwise a plain launch (rfi_last_launch).
 *   independent_launches  1 = a flagging launch that reads no byte that a flagging
 *                  launch still possibly running on the stream writes, and writes no
 *                  byte that one reads or writes (input, flags, statistics, averages,
 *                  weights, and the context state it uses: the open bin's carry when a
 *                  block starts or ends inside a bin, the open window's samples with
 *                  partial_windows, the thresholds' state with adaptive, the pending
 *                  hop with window_hop), does not wait for the kernel before it: its
 *                  blocks start their work while the launches before it drain.  For a
 *                  stream of blocks that each close their bins (K dividing T) written
 *                  into a ring of output buffers, consecutive launches overlap fully.
 *                  The caller promises that no kernel of its own that lets its
 *                  successor start early (griddepcontrol.launch_dependents,
 *                  cudaTriggerProgrammaticLaunchCompletion) writes a block's input or
 *                  reads its outputs between two calls on the stream; plain kernels,
 *                  copies and events in between need nothing.  Results are identical.
 *                  At most 32 launches are kept in flight; the next is a plain launch.
 *                  rfi_destroy, rfi_reset and rfi_set_state synchronise the device and
 *                  forget the launches made until then.  0 = off (default).
 *   window_hop     overlapping windows: a window of M samples starts every H =
 *                  window_hop samples (0 or M = no overlap, the paper's windows).
 *                  Only H = M/2 is built: every sample lies in two windows and is
 *                  flagged when either is.  A sample is final (flag known, averaged)
 *                  once the second window holding it has been evaluated, M - H samples
 *                  later, so a call returns the windows it completes (T/H, one fewer at
 *                  the stream's start), the flag bits of the samples that became final
 *                  (n_win * H bits from first_sample, see rfi_windows_for) and the bins
 *                  of K samples (K a multiple of H) that closed.  T must be a multiple of
 *                  H.  Needs time-only windows, float32 arithmetic, the direct loader,
 *                  the 128-register budget, plain stores, no Kahan summation and
 *                  lanes_per_row <= 4; excludes partial_windows and adaptive; a batch
 *                  takes it with contexts of the same hop and shape.  Any split of a
 *                  stream at multiples of H gives bit-identical results, alone or in a
 *                  batch.
 *   lane_split     0 = the lanes_per_row lanes of a row split every window's load
 *                  units (default).  1 = they take whole windows in turn (lane j the
 *                  stream's windows g with g mod P = j): no butterfly over the row's
 *                  lanes and one evaluation per window, for small windows and T x F
 *                  footprints, with P times shorter tasks than one lane per row.
 *                  lanes_per_row 2, 4 or 8 (P need not divide M), K/M >= lanes_per_row;
 *                  the direct loader, the 128-register budget (or max_registers = 96
 *                  for binary16 windows of odd length with 2 lanes: more resident
 *                  warps, the same results, batched with the 128-register kernel),
 *                  plain stores, no Kahan (precision = 1 with time-only windows: each
 *                  window still runs sample by sample in one lane, so its statistics
 *                  and flags equal those of the one-lane mixed kernel); excludes
 *                  partial_windows, adaptive and window_hop; a batch takes it with
 *                  contexts of the same split and shape.  Results differ from the
 *                  default split only in the order in which a bin's sums are added
 *                  (and the last bit of r's sum of squares).
 * The reduction order of a window depends only on (M, P, load unit), so two
 * contexts with the same shape give bit-identical results for the same data,
 * whether launched alone or inside a batch. */
typedef struct {
    int lanes_per_row;
    int warps_per_block;
    int host_max_T;
    int host_chunks;
    int compensated;
    int prefetch_bytes;
    int prefetch_groups;
    int max_registers;
    int window_F;
    int precision;
    int loader;
    int tma_stage_windows;
    int tma_stages;
    int debug_inject_wait_timeout;
    int buffered_stores;
    int partial_windows;
    int adaptive;
    int overlap_bytes;
    int window_hop;
    int lane_split;
    int independent_launches;
} rfi_options;

/* Parameters of the online SK thresholds (option `adaptive`). */
typedef struct {
    double alpha;     /* weight of a new clean window once n >= 1/alpha; 0 = plain mean */
    double k_sigma;   /* half width of the accepted interval in standard deviations */
    int n_warm;       /* clean windows a row needs before its own thresholds apply */
} rfi_adaptation;

/* Create a context for one stream of `stations` stations (B = N(N+1)/2 baselines)
 * and `channels` channels, window M = window_M >= 2 samples and output averaging
 * factor K = avg_K samples (K a multiple of M).  Allocates the device state on the
 * current CUDA device.  *out is set to NULL on failure. */
int rfi_create(rfi_ctx **out, int stations, int channels, int window_M, int avg_K,
               const rfi_thresholds *thr, rfi_dtype dtype);
int rfi_create_ex(rfi_ctx **out, int stations, int channels, int window_M, int avg_K,
                  const rfi_thresholds *thr, rfi_dtype dtype, const rfi_options *opt);

/* Rows R = B * C of the stream. */
int rfi_rows(const rfi_ctx *ctx, long long *rows);

/* Number of averaged outputs per row that the next rfi_process_block with T
 * samples will complete: floor((n_seen + T)/K) - floor(n_seen/K), where n_seen is
 * the number of samples already processed. */
int rfi_outputs_for(const rfi_ctx *ctx, int T, int *n_out);

/* Windows the next rfi_process_block with T samples will complete, n_win: the call
 * returns n_win statistics per row (footprint) and n_win M flag bits per row, bit i
 * for stream sample *first_sample + i (first_sample may be NULL).  Without
 * partial_windows, n_win = T/M and first_sample = n_seen.  With it, a window left
 * open by earlier blocks is completed first: n_win = (n_seen mod M + T) / M and
 * first_sample = n_seen - n_seen mod M (Sec. 2: windows of consecutive samples of a
 * stream, whatever the correlator's block length).  With overlapping windows (hop H),
 * E(n) = n >= M ? (n - M)/H + 1 : 0 windows are complete after n samples: n_win =
 * E(n_seen + T) - E(n_seen), n_win H flag bits per row, first_sample = E(n_seen) H. */
int rfi_windows_for(const rfi_ctx *ctx, int T, int *n_win, long long *first_sample);

/* The launch shape the context uses (after automatic choice). */
int rfi_get_options(const rfi_ctx *ctx, rfi_options *opt);

/* How the context's last single-stream flagging launch was ordered on its stream
 * (options overlap_bytes and independent_launches; no counterpart in the paper, a
 * diagnostic): *order = 2 independent (its blocks did not wait for the kernel before),
 * 1 waiting (they waited for it before touching memory), 0 plain (ordered after all
 * earlier work: overlap off, the staged loaders, or the launches in flight did not
 * allow either), -1 none yet or recorded into a CUDA graph. */
int rfi_last_launch(const rfi_ctx *ctx, int *order);

/* Replace the thresholds (takes effect for work issued afterwards). */
int rfi_set_thresholds(rfi_ctx *ctx, const rfi_thresholds *thr);

/* Adaptive contexts only (else RFI_EINVAL): set the parameters of the online SK
 * thresholds (0 <= alpha <= 1, finite k_sigma >= 0, n_warm >= 1), effective for work
 * issued afterwards; and copy the per-row state, float[R/F][4] = {n, mean of tau,
 * mean of tau^2, unused}, to (write = 0) or from (write = 1) a host buffer of at least
 * 4 R/F floats, after synchronising `stream`. */
int rfi_set_adaptation(rfi_ctx *ctx, const rfi_adaptation *p);
int rfi_adaptive_state(rfi_ctx *ctx, float *host, size_t n_floats, int write, void *stream);

/* Process one block of T samples (T a positive multiple of M, or any T with
 * partial_windows) of every row.  n_win = rfi_windows_for(T) windows complete.
 *   vis    [R][T][4 correlations][re, im] in the context's dtype; 32-byte aligned.
 *   flags  [R][ceil(n_win M/32)] uint32: bit (t mod 32) of word t/32 is 1 when sample
 *          t of the completed windows (t = 0 at first_sample; the block's own sample 0
 *          unless a window was open) lies in a flagged window (the flag applies to
 *          all 4 correlations).  Bits at t >= n_win M are 0.  4-byte aligned.
 *   avg    [R][n_out][4][re, im] float32: mean of the unflagged samples of every
 *          averaging bin that completes in this call (n_out = rfi_outputs_for);
 *          0 where every sample of the bin was flagged.  16-byte aligned.
 *   weight [R][n_out] float32: unflagged samples of the bin / K.
 *   stats  [3][R/F][n_win] float32: tau, r_Re, r_Im of every completed window (SoA;
 *          F = 1 unless the context has a T x F footprint).
 * avg and weight may be NULL only when n_out == 0, flags and stats only when n_win ==
 * 0.  Asynchronous on `stream`; allocates nothing and never synchronises, so a call can
 * be captured in a CUDA graph (the captured launch keeps this call's arguments: replay
 * it only where they repeat, e.g. K = T with whole windows; rfi_batch_graph_* updates
 * them per launch). */
int rfi_process_block(rfi_ctx *ctx, const void *vis, int T, uint32_t *flags, float *avg,
                      float *weight, float *stats, void *stream);

/* As rfi_process_block, but every buffer is in HOST memory (page-locked memory
 * lets the copies overlap).  Copies the block in through the context's device
 * staging (requires host_max_T >= T at create), runs the kernel per row chunk and
 * copies the outputs back; returns after the outputs are in host memory. */
int rfi_process_block_host(rfi_ctx *ctx, const void *vis, int T, uint32_t *flags,
                           float *avg, float *weight, float *stats, void *stream);

/* Process one block for each of n contexts (1 <= n <= 64) in ONE persistent launch.
 * All contexts must share dtype, M, lanes_per_row, Kahan summation and the kernel
 * variant (precision, partial_windows, adaptive) (else RFI_EINVAL); register budget,
 * buffered stores, prefetch and loader may differ (a batch runs the direct loader with
 * the 128-register budget and plain stores, prefetching as each context asks).  T[i],
 * sizes and layouts per context are as for
 * rfi_process_block.  Warps take (context, row group) tasks from a device counter
 * owned by ctxs[0]; two batches that share ctxs[0] must not run concurrently.  Results
 * are bit-identical to rfi_process_block on each context alone (Sec. 2: every
 * (baseline, channel) stream is flagged independently). */
int rfi_process_batch(rfi_ctx *const *ctxs, int n, const void *const *vis, const int *T,
                      uint32_t *const *flags, float *const *avg, float *const *weight,
                      float *const *stats, void *stream);

/* A batch captured once in a CUDA graph and replayed.  rfi_batch_graph_create
 * fixes the contexts and block lengths; each rfi_batch_graph_launch supplies this
 * step's buffers, updates the captured kernel's parameters (no allocation) and
 * launches the graph on `stream`. */
typedef struct rfi_batch_graph rfi_batch_graph;
int rfi_batch_graph_create(rfi_batch_graph **out, rfi_ctx *const *ctxs, int n, const int *T);
int rfi_batch_graph_launch(rfi_batch_graph *g, const void *const *vis, uint32_t *const *flags,
                           float *const *avg, float *const *weight, float *const *stats,
                           void *stream);
int rfi_batch_graph_destroy(rfi_batch_graph *g);

/* ---- Entry point that allocates nothing ------------------------------------
 * The paper has no counterpart; this serves callers that may not allocate device
 * memory -- e.g. a pipeline stage whose GPU memory is reserved up front by its own
 * pool, or a real-time thread that cannot risk the implicit synchronisation of an
 * allocation.  They pass their own inputs and outputs; the only working memory, the
 * carry of each row's open averaging bin, lives in a fixed device array of
 * RFI_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until exit.
 *
 * rfi_process_block_noalloc processes one block like rfi_process_block, without a
 * context: geometry, thresholds and dtype come with every call, and n_seen is the
 * number of samples of this stream processed before the block (a multiple of M).
 * Buffers, layouts and alignment are those of rfi_process_block.  The kernel uses
 * one lane per row, so results equal rfi_process_block on a context created with
 * lanes_per_row = 1 and otherwise default options.
 *   - Limit: R * 36 bytes of carry must fit the array, i.e. at most
 *     RFI_NOALLOC_SCRATCH_BYTES / 36 = 116508 rows; larger streams get RFI_EINVAL.
 *   - The first call made in each CUDA context (the device's primary context, or a
 *     context the caller made current through the driver API; after cudaDeviceReset
 *     the new primary context counts as another) looks up the array's device address
 *     with cudaGetSymbolAddress (which may load the module) and keeps it for that
 *     context; make that first call before any stream capture.
 *   - Blocks with T * R > 2^40 samples get RFI_EINVAL, as for rfi_process_block.
 *   - Every call shares the array, and it keeps what the last call wrote.  A block
 *     that continues an open bin (n_seen % K != 0) reads the carry left by the
 *     previous call, so such blocks of one stream must follow each other with no
 *     call for another stream in between.  Calls that overlap on the GPU race.
 *   - Its kernel lets the launch after it start early; the call counts its launch
 *     (without allocating) under the lock that orders the library's flagging launches,
 *     so that the next flagging launch of a context, on any stream, waits for the
 *     launch before it (or runs in plain stream order) rather than starting
 *     independently (option independent_launches).
 *   - Calls no cudaMalloc, cudaFree or other allocating routine. */
#define RFI_NOALLOC_SCRATCH_BYTES (4u << 20)
int rfi_process_block_noalloc(int stations, int channels, int window_M, int avg_K,
                              const rfi_thresholds *thr, rfi_dtype dtype, long long n_seen,
                              const void *vis, int T, uint32_t *flags, float *avg,
                              float *weight, float *stats, void *stream);

/* Checkpoint and resume.  A stream's state is its sample count, thresholds and the
 * per-lane running sums of every row's open averaging bin (and, with
 * partial_windows, the raw samples of every row's open window; with adaptive, the
 * running moments of tau and their parameters).  rfi_get_state
 * synchronises `stream` and copies the state into a caller-owned host buffer of
 * rfi_state_size bytes (a plain byte blob); rfi_set_state loads it into a context of
 * the same geometry and launch shape (rows, lanes_per_row, M, K, window_F, dtype,
 * partial_windows, adaptive; else
 * RFI_EINVAL), after which the stream continues exactly (bit for bit) where the saved
 * one stopped. */
int rfi_state_size(const rfi_ctx *ctx, size_t *bytes);
int rfi_get_state(rfi_ctx *ctx, void *buf, size_t bytes, void *stream);
int rfi_set_state(rfi_ctx *ctx, const void *buf, size_t bytes);

/* Synchronise `stream` and report a device-side failure of work issued for the
 * context: RFI_ETIMEOUT when a bounded wait in the kernel gave up (the context then
 * stays failed until rfi_reset), RFI_OK otherwise. */
int rfi_check(rfi_ctx *ctx, void *stream);

/* Drop the averaging carry and the sample count (stream restart); clears a sticky
 * error.  Synchronises with work already issued for the context. */
int rfi_reset(rfi_ctx *ctx);

/* Free the context and its device state.  rfi_destroy(NULL) is a no-op. */
int rfi_destroy(rfi_ctx *ctx);

/* Static description of a status code. */
const char *rfi_status_str(int status);

/* Text of the last error recorded by the library on the calling thread. */
const char *rfi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RFI_H */
