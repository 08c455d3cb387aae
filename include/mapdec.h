/*
 * mapdec.h -- C ABI of libmapdec.so, a GB300 (sm_103a) MAP decoder for the
 * Davey-MacKay binary substitution/insertion/deletion (BSID) channel.
 *
 * The decoder computes, for a frame of N q-ary symbols each sent as an n-bit
 * codeword C(D) and received as rho bits Y through the BSID channel
 * (Briffa, "GPU Implementation and Optimization of a Flexible MAP Decoder for
 * Synchronization Correction", Sec. II):
 *   (1) the receiver metric R(Y[p .. p+j) | C(D)) for every start p, codeword D
 *       and received length j, by the lattice of eqs. (F), (F_lastrow) with at
 *       most I insertions before each transmitted bit;
 *   (2) gamma_i(m', m, D) = Pr{D_i = D} R(...) (eq. gamma) and the forward and
 *       backward recursions of eqs. (alpha), (beta) with per-index
 *       normalisation (eqs. alpha_norm, alpha_prenorm);
 *   (3) the a-posteriori probabilities L_i(D) of eqs. (L), (lambda), (sigma),
 *       normalised over D for every symbol;
 *   (4) the frame log-likelihood log P(Y) = sum_i log c_i + log alpha_N(rho-tau),
 *       c_i the forward normalisers of eq. (alpha_norm).
 * Gradients of log P(Y) (not in the paper) are provided by an adjoint path,
 * and extrinsic outputs for iterative decoding with an outer code (Sec. II-A:
 * eq. (L) without each symbol's own prior) by mapdec_decode_ext and
 * mapdec_batch_decode_ext.
 *
 * Conventions shared by every entry point
 *   - Drift states m lie in [-xmax, xmax] at symbol boundaries; the drift
 *     change over one symbol lies in [-n, n*I].  The frame is isolated and its
 *     received length rho is known: alpha_0 = [m = 0], beta_N = [m = rho - tau],
 *     tau = n*N.  |rho - tau| must not exceed xmax.
 *   - Bits are passed one per byte (0 or 1).  A codebook is q*n bytes,
 *     row D = C(D) = (x_1 .. x_n); rows must be distinct (the encoding is
 *     injective, Sec. II-A).
 *   - Priors are N*q floats, row i = Pr{D_i = .}, entries >= 0, each row with a
 *     positive sum; they are used as given (not renormalised).  NULL means
 *     uniform 1/q.
 *   - Arithmetic: FP32 for the lattice, gamma, alpha, beta and APPs; FP64 for
 *     the sum of log normalisers and for gradient reductions.
 *   - Every data pointer may be host or device memory (detected per call).
 *     Pinned (page-locked) host buffers of at least 1 MiB whose address is a
 *     multiple of 16 bytes are read or written by a copy kernel through their
 *     device mapping; other host buffers by the copy engine (pageable memory
 *     is staged by the driver and is much slower).
 *     The caller owns all buffers; a handle owns its device scratch.
 *     Work is issued on the handle's stream.  mapdec_decode,
 *     mapdec_decode_ext, mapdec_loglik_grad, mapdec_receiver_metric,
 *     mapdec_batch_decode, mapdec_batch_decode_ext and
 *     mapdec_batch_loglik_grad return after that stream has drained, so
 *     their status covers the whole computation; mapdec_batch_run is
 *     asynchronous.
 *   - There is no CPU fallback: if no CUDA device is usable the calls fail
 *     with MAPDEC_ERR_CUDA.
 *   - A handle must not be used from two threads at once.
 *   - Every call returns a status; mapdec_strerror() names it.
 */
#ifndef MAPDEC_H
#define MAPDEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MAPDEC_OK = 0,
    MAPDEC_ERR_ARG = 1,         /* invalid argument (sizes, probabilities, codebook) */
    MAPDEC_ERR_DRIFT_RANGE = 2, /* |rho - tau| > xmax */
    MAPDEC_ERR_ZERO_PROB = 3,   /* no channel path within the drift limits explains Y */
    MAPDEC_ERR_NOMEM = 4,       /* device or host allocation failed */
    MAPDEC_ERR_CUDA = 5,        /* CUDA runtime error or no usable device */
    MAPDEC_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    MAPDEC_ERR_UNSUPPORTED = 7, /* parameters outside what the kernels support */
    MAPDEC_ERR_TOO_LARGE = 8    /* frame's scratch exceeds mapdec_decode_noalloc's arena */
};

typedef struct mapdec mapdec_t;

/*
 * Create a decoder for one code and channel (Sec. II-A, II-B).
 *   q >= 2 codewords of n bits (1 <= n <= 31, q <= 2^n, n*(I+1) <= 63),
 *   codebook: q*n bytes (host or device), distinct rows;
 *   N >= 1 symbols per frame; channel Pi, Pd, Ps with Pi, Pd, Ps >= 0,
 *   Pi + Pd < 1, Ps <= 1; insertion cap I >= 1; drift limit xmax >= 0.
 * Plans the tiles and allocates the device scratch of the decode path once,
 * for the largest admissible received length rho_max = tau + xmax (tau = n*N);
 * mapdec_decode and mapdec_decode_ext then reuse it for every received length
 * in [tau - xmax, tau + xmax] without allocating.  The gradient path's scratch
 * is allocated by the first mapdec_loglik_grad call, and the output buffer of
 * mapdec_receiver_metric by its first call, each once for rho_max.
 * On success *out holds the handle (destroy with mapdec_destroy).
 */
int mapdec_create(mapdec_t **out, int q, int n, const uint8_t *codebook, int N, double Pi,
                  double Pd, double Ps, int I, int xmax);

/* Issue all work of this handle on `cuda_stream` (a cudaStream_t; NULL = default stream). */
int mapdec_set_stream(mapdec_t *h, void *cuda_stream);

/*
 * Decode one frame: steps (1)-(4) above.
 *   rx: rx_len received bits (one per byte); priors: N*q floats or NULL;
 *   app_out: N*q floats, row i = L_i(.), sums to 1;  loglik_out: 1 double.
 * Either output may be NULL.  Returns MAPDEC_ERR_DRIFT_RANGE if
 * |rx_len - n*N| > xmax, MAPDEC_ERR_ZERO_PROB if P(Y) = 0 within the limits.
 * The call returns after the work has completed on the handle's stream (the
 * status of the decode is known only then).
 */
int mapdec_decode(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                  float *app_out, double *loglik_out);

/*
 * mapdec_decode plus the extrinsic outputs of the frame (see
 * MAPDEC_BATCH_EXTRINSIC): ext_out N*q floats, row i = E_i(.), sums to 1.
 * Any output may be NULL.
 */
int mapdec_decode_ext(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                      float *app_out, float *ext_out, double *loglik_out);

/*
 * log P(Y) and its gradient (the adjoint path; not in the paper):
 *   dlogp_dchan[0..2] = d logP / d(Pi, Pd, Ps), with Pt = 1 - Pi - Pd and the
 *     drift limits held fixed (FP64);
 *   dlogp_dpriors: N*q floats, d logP / d Pr{D_i = D};
 *   loglik_out: log P(Y).
 * Requires Pd > 0 and Pt*(1-Ps) > 0.  Any output may be NULL.
 */
int mapdec_loglik_grad(mapdec_t *h, const uint8_t *rx, int64_t rx_len, const float *priors,
                       double *dlogp_dchan, float *dlogp_dpriors, double *loglik_out);

/*
 * Step (1) alone: R_out[(p*q + D)*(n*(I+1)+1) + j] = R(Y[p .. p+j) | C(D)) for
 * p = 0..rx_len, D < q, j = 0..n*(I+1); entries with p + j > rx_len are 0.
 * R_out holds (rx_len+1)*q*(n*(I+1)+1) floats.
 */
int mapdec_receiver_metric(mapdec_t *h, const uint8_t *rx, int64_t rx_len, float *R_out);

/*
 * Stream decoding with a single-frame handle: set (or, with NULL, clear) the
 * drift priors of the frame's start and end (2*xmax+1 floats each, host or
 * device; see mapdec_frame_desc_t.drift_start / drift_end) used by the
 * following mapdec_decode, mapdec_decode_ext and mapdec_loglik_grad calls.
 * The values are copied into buffers the handle allocated at create; nothing
 * is allocated.  MAPDEC_ERR_ARG for negative or non-finite entries or an
 * all-zero prior.
 */
int mapdec_set_drift_priors(mapdec_t *h, const float *drift_start, const float *drift_end);

/* Release a handle and its device scratch (NULL is ignored). */
void mapdec_destroy(mapdec_t *h);


/* Static string for a status code. */
const char *mapdec_strerror(int status);

/* ------------------------------------------------------------------------ */
/* Batched decoding of many frames with different codes and channels         */
/* ------------------------------------------------------------------------ */

/* One frame of a batch: its code, channel, drift limit and received length. */
typedef struct {
    int q, n, N, I, xmax;
    double Pi, Pd, Ps;
    const uint8_t *codebook; /* q*n bytes, host or device; copied at create */
    int64_t rx_len;          /* rho of this frame */
    int codebook_per_symbol; /* 0: one codebook for every symbol; 1: one per symbol
                                (the constituent encodings C_i of Sec. II-A):
                                codebook holds N*q*n bytes, symbol i's q*n at offset
                                i*q*n, each with distinct rows; q <= 256.  The
                                receiver metric then depends on the symbol, so the
                                producers evaluate the paper's (i, m', D) grid of
                                lattices (no position dedupe): about M/n times the
                                work of one codebook.  Not with
                                MAPDEC_BATCH_SEGMENTED or mapdec_decode_noalloc
                                (MAPDEC_ERR_UNSUPPORTED). */
    const float *drift_start;  /* stream decoding (Sec. II-C: alpha_0 and beta_N are the
                                  priors of the frame boundaries): 2*xmax+1 floats, entry
                                  m + xmax = Pr{the frame starts at received position m},
                                  host or device, copied at create; NULL: the frame
                                  starts at position 0 (alpha_0 = [m = 0]).  Mass at
                                  m < 0 carries no path (no received bits there). */
    const float *drift_end;    /* 2*xmax+1 floats, entry m + xmax = Pr{the frame ends
                                  at received position tau + m}; received bits after
                                  the end belong to the next frame.  NULL: the frame
                                  ends at rx_len (beta_N = [m = rx_len - tau]).  With
                                  boundary priors log P(Y) = log sum over both
                                  boundaries of prior x likelihood of the piece between
                                  them, and the APPs are the matching mixture.
                                  Entries >= 0, finite, some positive; else
                                  MAPDEC_ERR_ARG.  Not with mapdec_decode_noalloc. */
} mapdec_frame_desc_t;

/*
 * Decode one frame without allocating any memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate once
 * running -- a receive pipeline whose memory is fixed at start-up, a host
 * framework that owns every device allocation, real-time code that must not
 * risk a cudaMalloc blocking, fragmenting or failing mid-stream.
 *   frame: code, channel, drift limit and rx_len of the frame; its codebook
 *     (q*n bytes) may be host or device memory.  q <= 64.
 *   rx_dev (rx_len bytes), priors_dev (N*q floats, or NULL for uniform 1/q),
 *   app_dev (N*q floats), loglik_dev (1 double): device memory owned by the
 *   caller.
 *   cuda_stream: a cudaStream_t (NULL = default stream).
 * Results equal mapdec_decode's.  All scratch lives in one static device
 * array of 32 MiB per GPU that loads the library, held until the process
 * exits; a frame whose scratch does not fit is rejected with
 * MAPDEC_ERR_TOO_LARGE (about N * (2 xmax + 1) * (n(I+1)+1) * 4 bytes for the
 * transition sums dominates).  The first call on a device looks up the
 * array's address on that device; make that first call before any stream
 * capture.  Every call shares the array and leaves its contents behind (the
 * next call clears what must start at zero), so calls whose work overlaps on
 * the GPU -- concurrent streams, threads or devices sharing a context -- race
 * and must be serialised by the caller.  The call returns after the stream
 * has drained, with the decode's status.
 */
int mapdec_decode_noalloc(const mapdec_frame_desc_t *frame, const uint8_t *rx_dev,
                          const float *priors_dev, float *app_dev, double *loglik_dev,
                          void *cuda_stream);

/* batch flags */
enum {
    MAPDEC_BATCH_GRAPH = 1,  /* capture the launch sequence in a CUDA graph */
    MAPDEC_BATCH_PLAIN = 2,  /* one frame per launch, default tile sizes, no graph */
    MAPDEC_BATCH_GRAD = 4,   /* allocate for mapdec_batch_loglik_grad */
    MAPDEC_BATCH_TIMING = 8, /* record CUDA events at phase boundaries of every run */
    /*
     * Checkpoint and recompute (not in the paper, which keeps every forward
     * and backward row of Sec. II-C in memory): each frame is cut into
     * segments of K = ceil(sqrt(N)) symbols (environment MAPDEC_SEG_K
     * overrides K).  A first sweep runs the forward recursion segment by
     * segment, keeping only the row at every segment boundary and the tilt
     * record; a second sweep, last segment first, recomputes the segment's
     * transition weights and forward rows from its checkpoint (the same rows,
     * bit for bit) beside the backward recursion, then the APPs of that
     * segment.  Scratch per frame falls from O(N) rows to O(K + N/K) rows at
     * the price of computing the transition weights twice.  Results equal
     * the unsegmented run's to rounding order of the APP partial sums.
     */
    MAPDEC_BATCH_SEGMENTED = 16,
    /*
     * Also produce extrinsic outputs (mapdec_batch_decode_ext): for iterative
     * decoding with an outer code (Sec. II-A) the inner decoder passes on
     * what it learned about each symbol from the received sequence and the
     * other symbols, i.e. eq. (L) without the symbol's own prior:
     *   E_i(D) = sum_{m', m} alpha_i(m') R(Y[n i + m' .. n(i+1) + m) | C(D)) beta_{i+1}(m),
     * normalised over D.  The APP is the prior times E_i, renormalised.
     */
    MAPDEC_BATCH_EXTRINSIC = 32
};

typedef struct mapdec_batch mapdec_batch_t;

/*
 * Plan a batch: frames[0..num_frames).  Validates every frame (as
 * mapdec_create plus |rx_len - n*N| <= xmax), chooses tile sizes (from the
 * tuning table if one was loaded), allocates device scratch within
 * `mem_budget_bytes` (0 = 60% of free device memory; frames are processed in
 * waves that fit) and the batch's own device input/output buffers.
 * Frame f's bits, priors and APPs sit in concatenated buffers at the offsets
 * reported by mapdec_batch_layout.
 */
int mapdec_batch_create(mapdec_batch_t **out, const mapdec_frame_desc_t *frames, int num_frames,
                        int flags, int64_t mem_budget_bytes);

/*
 * Offsets of frame f in the concatenated buffers (host arrays of num_frames):
 * rx_offsets[f] (bytes), sym_offsets[f] (rows of q floats, i.e. priors and
 * APPs of frame f start at element sym_offsets[f]).  Also the totals.
 */
int mapdec_batch_layout(mapdec_batch_t *b, int64_t *rx_offsets, int64_t *sym_offsets,
                        int64_t *rx_total, int64_t *prior_elems_total);

/*
 * Device pointers of the batch's resident input/output buffers, so callers
 * can fill inputs in place and run without copies (any may be NULL).
 */
int mapdec_batch_buffers(mapdec_batch_t *b, uint8_t **rx_dev, float **priors_dev,
                         float **app_dev, double **loglik_dev);

/*
 * Byte offset of frame f's bits inside the resident rx buffer returned by
 * mapdec_batch_buffers (the same dense concatenation as mapdec_batch_layout's
 * rx_offsets); -1 if f is out of range.
 */
int64_t mapdec_batch_rx_offset(mapdec_batch_t *b, int frame);

/*
 * Decode the resident inputs into the resident outputs.  Stream-ordered and
 * asynchronous: call mapdec_batch_sync (or synchronise the stream) before
 * reading the outputs.
 */
int mapdec_batch_run(mapdec_batch_t *b);

/* Wait for the batch's stream; returns the worst per-frame status of the last run. */
int mapdec_batch_sync(mapdec_batch_t *b);

/* Per-frame status of the last run (host array of num_frames ints; synchronous). */
int mapdec_batch_status(mapdec_batch_t *b, int *status_per_frame);

/*
 * Decode all frames: copies rx_all / priors_all (host or device; priors_all
 * may be NULL = uniform) into the resident buffers, runs, and copies APPs and
 * log-likelihoods to app_all / loglik_all (host or device, may be NULL).
 * Passing the batch's own resident buffers (mapdec_batch_buffers) as inputs
 * skips their copy.
 */
int mapdec_batch_decode(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                        float *app_all, double *loglik_all);

/*
 * As mapdec_batch_decode, plus the extrinsic outputs (batch created with
 * MAPDEC_BATCH_EXTRINSIC, else MAPDEC_ERR_ARG): ext_all like app_all, row i
 * of frame f = E_i(.) of that frame, summing to 1 (host or device, may be
 * NULL).  E_i is defined where the prior is 0.
 */
int mapdec_batch_decode_ext(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                            float *app_all, float *ext_all, double *loglik_all);

/*
 * Gradients for every frame (batch created with MAPDEC_BATCH_GRAD):
 * dchan_all[3*f + k] = d logP_f / d(Pi, Pd, Ps)_k, dpriors_all like app_all.
 * Inputs as for mapdec_batch_decode.
 */
int mapdec_batch_loglik_grad(mapdec_batch_t *b, const uint8_t *rx_all, const float *priors_all,
                             double *dchan_all, float *dpriors_all, double *loglik_all);

/* Issue the batch's work on `cuda_stream` (a cudaStream_t; NULL = default stream). */
int mapdec_batch_set_stream(mapdec_batch_t *b, void *cuda_stream);

/* Release a batch, its CUDA graph and all its device buffers (NULL is ignored). */
void mapdec_batch_destroy(mapdec_batch_t *b);

/*
 * Number of kernel launches the last run issued (graph nodes count as
 * launches).  For accounting in benchmarks.
 */
int64_t mapdec_batch_last_launches(mapdec_batch_t *b);

/*
 * Device time of each phase of the last run, summed over waves (batch created
 * with MAPDEC_BATCH_TIMING; synchronises the stream).  ms[0..4] = received-bit
 * packing, forward producers (lattice + W), forward/backward chains, backward
 * producers (lattice + APP sums), finalize.  When frames need several waves,
 * one wave's chains run on a second stream while other waves' producers run,
 * so the phase times overlap and their sum exceeds the run's wall time.  In
 * a MAPDEC_BATCH_SEGMENTED batch ms[1] is the whole recording sweep, ms[3]
 * the whole recompute sweep and ms[2], ms[4] are 0.
 */
int mapdec_batch_phase_ms(mapdec_batch_t *b, double *ms);

/*
 * Tuning table (not in the paper, which picks its block sizes by a run-time
 * rule): launch parameters per (q, n, I) class, applied to batches created
 * afterwards (not to MAPDEC_BATCH_PLAIN batches).  A zero field keeps the
 * planner's choice; values that do not fit the device are replaced by the
 * planner's choice.  The table is process-wide and guarded by a mutex.
 */
typedef struct {
    int P;               /* received positions per producer tile */
    int nsub;            /* producer tiles per APP super-tile */
    int chain_budget_kb; /* shared memory of one recursion CTA, 16..220 KB */
    int chain_stages;    /* bulk-copy stages in flight in the recursions, 2..8 */
    int store_metric;    /* 1: keep the receiver metrics R in device memory between the
                            forward and APP producers (decode only; about
                            (rho+1) * roundup4(q) * (n(I+1)+1) * 4 bytes per frame);
                            0 or -1: recompute them */
    int tensor_cores;    /* 0: the planner's rule (the forward producer on the tensor
                            cores for frames whose tiles span at least 36 symbols,
                            the APP producer on the CUDA cores); 1: both producers on
                            the tensor cores wherever the class supports them (see
                            mapdec_batch_tc_frames); 2: FP32 CUDA-core producers */
    int chain_threads;   /* block size of the recursion kernel: 128, 256 or 512
                            (0 = 256); the batch takes the value of its last frame
                            whose class sets it */
} mapdec_tune_t;

/* Set (t != NULL) or remove (t == NULL) the entry of class (q, n, I). */
int mapdec_tune_set(int q, int n, int I, const mapdec_tune_t *t);
/* Copy the entry of class (q, n, I) to *t; MAPDEC_ERR_ARG if there is none. */
int mapdec_tune_get(int q, int n, int I, mapdec_tune_t *t);
/* Remove every entry. */
int mapdec_tune_clear(void);

/* Number of waves the batch's frames were split into (scratch budget). */
int mapdec_batch_num_waves(mapdec_batch_t *b);

/*
 * Frames whose contractions run on the tensor cores (tcgen05, bf16 operands
 * split into high and low parts, FP32 accumulation; an implementation choice,
 * not in the paper).  The planner picks the forward producer's for decode
 * batches, classes with q a multiple of 16 up to 64 and n >= 4 whose tiles fit
 * and span at least 36 symbols (MAPDEC_TC_MIN_S overrides the count); the
 * other frames, and every frame of a MAPDEC_BATCH_GRAD batch, use the FP32
 * CUDA-core producers.  The environment variables, read when a batch is
 * created: MAPDEC_TC=0 keeps every producer on the CUDA cores, MAPDEC_TC=1
 * puts both producers on the tensor cores wherever supported, MAPDEC_TC_BWD
 * switches the APP producer's choice on (1) or off (0).  If flags is not NULL it receives one int per frame: bit 0
 * set when the forward producer (W contraction) runs on the tensor cores,
 * bit 1 when the APP producer does.  Returns the number of frames with bit 0
 * set, or -1 for a NULL batch.
 */
int mapdec_batch_tc_frames(mapdec_batch_t *b, int *flags);

/*
 * Measured FP32 FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA), the arithmetic roof the decoder's kernels are reported against.  Not
 * part of the paper's method.  Runs a short probe kernel (tens of
 * milliseconds) on `cuda_stream` (NULL = legacy default stream) and waits for
 * it.  Returns MAPDEC_ERR_ARG for a NULL output, MAPDEC_ERR_NOMEM or
 * MAPDEC_ERR_CUDA on failure (the output is then 0).
 */
int mapdec_fp32_fma_peak(double *tflops_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MAPDEC_H */
