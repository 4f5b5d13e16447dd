/*
 * tsx.h -- C ABI of the GB300 trapping-set enumeration library.
 *
 * The library implements the data-parallel hot path of the modified Cole
 * importance-sampling method (V. Usatyuk, arXiv 2208.05795, Sec. III):
 * impulse-perturbed message-passing decodes of the all-zero codeword on a
 * QC-LDPC (or general LDPC) Tanner graph, a bisection on the impulse
 * amplitude, extraction of the failing pattern's cycle-closed core as an
 * (a,b) trapping set, reduction to one canonical form per circulant-shift
 * orbit, and deduplication.  Every step runs in CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *   - The return value is TSX_OK (0) or a negative TSX_E* status; no
 *     exception or process exit crosses this boundary.
 *   - Input arrays are borrowed for the duration of the call and copied
 *     where they are kept; output objects are owned by the library until
 *     the matching free_* call.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Host pointers are plain pageable or pinned memory.
 *   - Calls on one object are not thread-safe; distinct objects may be used
 *     from distinct threads.
 */
#ifndef TSX_H
#define TSX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TSX_API __attribute__((visibility("default")))
#else
#define TSX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TSX_OK 0
#define TSX_EINVAL (-1)       /* bad argument or malformed code description */
#define TSX_ENOMEM (-2)       /* device or host allocation failed, or a table overflowed */
#define TSX_ECUDA (-3)        /* a CUDA runtime call failed */
#define TSX_ETIMEDOUT (-4)    /* a bounded device-side wait ran out */
#define TSX_EBUSY (-5)        /* resource in use (server admission) */
#define TSX_EUNSUPPORTED (-6) /* a degree or size above the compiled limits */
#define TSX_ENOTFOUND (-7)    /* unknown job id */
#define TSX_EAGAIN (-8)       /* job not finished yet */

/* Human-readable text for a status code (static storage). */
TSX_API const char *tsx_strerror(int status);

/* Compiled limits. */
#define TSX_MAX_DC 32    /* check-node degree */
#define TSX_MAX_DV 16    /* variable-node degree */
#define TSX_MAX_NB 64    /* QC base-matrix columns */
#define TSX_MAX_N 32767  /* variable nodes per code */

/* ---- codes (Sec. II, eqs. 1-3) --------------------------------------- */
typedef struct tsx_code tsx_code;

enum { TSX_CODE_QC = 0, TSX_CODE_CSR = 1 };

/* Description of a parity-check matrix.
 *   QC (eqs. 1-3): `shifts` is the m_b x n_b exponent matrix E(H),
 *     row-major, entries in {-1, 0, ..., Z-1}; -1 is the zero block and
 *     a >= 0 the circulant P^a whose row r has its 1 in column (r+a) mod Z.
 *     Variable node j*Z+k, check node i*Z+r.  Orbit representatives of the
 *     circulant-shift automorphism are the variable nodes j*Z.
 *   CSR: a general matrix by rows: row_ptr[m+1], col_idx[row_ptr[m]] with
 *     the variable nodes of each check, no duplicates.  No automorphism is
 *     used: every variable node is a representative. */
typedef struct {
    int32_t kind;           /* TSX_CODE_QC or TSX_CODE_CSR */
    int32_t m_b, n_b, Z;    /* QC */
    const int32_t *shifts;  /* QC, host */
    int32_t n, m;           /* CSR */
    const int32_t *row_ptr; /* CSR, host */
    const int32_t *col_idx; /* CSR, host */
} tsx_code_desc;

typedef struct {
    int32_t kind, n, m, E, Z, n_b, m_b;
    int32_t dv_max, dc_max;
    int32_t girth;       /* 0 if the graph has no cycle */
    int32_t n_rep;       /* orbit representatives */
    int64_t ball_total;  /* sum of the representatives' Tanner-ball sizes */
    int64_t device_bytes;
} tsx_code_info;

/* Validates `desc`, builds the device-resident tables (edge layout, Tanner
 * balls of the representatives: the variable layers of the depth-3
 * unrolled tree of Sec. III / Fig. 3) and computes the girth.  Blocks until
 * the tables are resident.  Errors: TSX_EINVAL (shift outside
 * {-1..Z-1}, index outside [0,n), duplicate edge, empty code),
 * TSX_EUNSUPPORTED (degree, n_b or n above the limits), TSX_ENOMEM,
 * TSX_ECUDA. */
TSX_API int load_code(const tsx_code_desc *desc, void *stream, tsx_code **out);
TSX_API void free_code(tsx_code *code);
TSX_API int code_info(const tsx_code *code, tsx_code_info *info);

/* ---- cycles and EMD spectrum (Sec. II, Prop. 1, Tables II and V) ---- */
/* Cycles of length 4 and 6 through every variable node (computed once by
 * load_code(): Table V's cycle densities per node).  c4, c6: host arrays of
 * n entries.  Errors: TSX_EINVAL. */
TSX_API int cycle_counts(const tsx_code *code, int64_t *c4, int64_t *c6);

/* The EMD spectrum of Sec. II (Table II).  A cycle of length 2l is an
 * exponent chain that closes (Prop. 1, eq. 3): a closed walk
 * v0 - c1 - v1 - ... - c_l - v0 of the Tanner graph that never steps straight
 * back (consecutive checks differ, consecutive variable nodes differ, c_l !=
 * c_1), taken up to rotation and reversal; it may pass a node twice (the
 * 4-cycle walked twice is an 8-cycle).  Its EMD is the number of checks
 * connected to exactly one of its variable nodes.  The walks are enumerated
 * from the orbit representatives (QC: the column index of a node is the
 * running alternating sum of the exponents, and a walk closes when it is
 * 0 mod Z) for l = 2 .. lmax (lmax <= 6).  count2l[l][e] / (2l) is the
 * number of cycles of length 2l with EMD e -- per circulant orbit for a QC
 * code (Table II's count "without multiplication by graph automorphism"), a
 * plain count for a general code; it is fractional for a cycle invariant
 * under part of the shift group.  walks[l]: closed walks from the
 * representatives.  Synchronizes `stream`; allocates a few KB.  Errors:
 * TSX_EINVAL (lmax), TSX_EUNSUPPORTED (search above ~4e11 walk steps),
 * TSX_ENOMEM, TSX_ECUDA. */
typedef struct {
    int32_t lmax;
    int64_t walks[7];
    int64_t count2l[7][128];
    double ms;             /* device time of the search (CUDA events) */
} tsx_emd_spectrum;
TSX_API int emd_spectrum(tsx_code *code, int32_t lmax, void *stream, tsx_emd_spectrum *out);

/* ---- trapping-set enumeration (Sec. III) ----------------------------- */
typedef struct tsx_ts_list tsx_ts_list;

enum {
    TSX_DEC_NMS_I16 = 0, /* fixed-point normalized min-sum, int16 messages */
    TSX_DEC_NMS_I8 = 1,  /* the same decoder with int8 check-to-variable storage (sat <= 169) */
    TSX_DEC_SPA_F32 = 2  /* single-precision sum-product */
};

typedef struct {
    int32_t decoder;     /* TSX_DEC_* */
    int32_t K;           /* maximum iterations (flooding schedule) */
    int32_t base_llr;    /* channel LLR of every bit, fixed point, units of 1/8 (> 0) */
    int32_t sat;         /* min-sum message and channel saturation (511 for int16) */
    int32_t alpha_num;   /* min-sum normalization (alpha_num * m) >> alpha_shift */
    int32_t alpha_shift;
    int32_t amp_steps;   /* s: amplitude range [0, 2^s - 1] (min-sum) or s halvings of [0,1] (sum-product) */
    float spa_clip;      /* sum-product channel/message clip (30) */
    float spa_amax;      /* sum-product impulse amplitude at eps = 1, LLR units (64) */
    int32_t max_size;    /* candidate sets: 1..4 nodes from a representative's Tanner ball */
    int32_t cycle_len;   /* 0, or 2l in 6..8: add the VN sets of 2l-cycles through the
                            representatives when l > max_size */
    int32_t record_candidates; /* 1: keep per-candidate records */
    int64_t cand_begin;  /* decode candidates [cand_begin, cand_end) of the canonical list */
    int64_t cand_end;    /* -1 = to the end */
    int32_t warps_per_cta; /* warps per codeword group (0 = automatic) */
    int32_t ctas_per_sm;   /* 0 = as many as are resident */
    int32_t kernel;        /* min-sum kernel: 0 automatic, 1 one codeword per group,
                              2 two codewords per lane (16-bit halves).  Automatic and 2 use
                              two codewords per lane where its 16-bit bounds hold and its
                              layout fits a CTA (for int16 QC codes of check degree > 8 whose
                              two posterior buffers do not fit: one buffer rebuilt by a
                              variable-node pass), else one codeword per group; the results
                              are the same */
    int32_t list_mode;     /* 1 (min-sum decoders): the ordered list of Sec. III -- every non-empty
                              S1(x_k) = Tree(X_k) and S2(x_k) = Tree(TS(X_k)), X_k = supp(x_k) u I,
                              of the decode at the threshold amplitude, k = kstart .. K_last, is a
                              trapping set; per set, count = candidates whose list holds it (each
                              candidate counted once) and flags bits 1-2 = which of S1 / S2 gave it.
                              Run as a second stage over the failing candidates only; per candidate
                              cand_ts = -1 and cand_flags = 0.  K <= 1000. */
    int32_t kstart;        /* list mode: first iteration of the list; 0 = max(1, floor(girth/2)),
                              -1 = ceil(average iterations of the decodes of the first stage that
                              converged to the all-zero word) (at least 1), > 0 as given */
    int32_t budget_wref;   /* 0: every candidate gets K iterations.  > 0: cycle-density budget --
                              candidate I gets K(I) = kmin + ceil((K - kmin) wref / (wref + W(I)))
                              iterations, W(I) = sum over v in I of 2 c4(v) + c6(v), c4 / c6 the 4- and
                              6-cycles through v (Sec. III, Table V) */
    int32_t budget_kmin;   /* the smallest budget (1 <= kmin <= K; K <= 65535 with a budget) */
} tsx_enum_params;

/* Fills `p` with the defaults: NMS int16, K=20, base 16, sat 511, alpha 3/4,
 * s=10, clip 30, amax 64, max_size 3, no cycle sets, records on, all
 * candidates, autotuned tile. */
TSX_API void enum_params_default(tsx_enum_params *p);

/* Runs the whole hot path for `code` on `stream`: candidate generation and
 * canonical dedupe, the impulse decodes with amplitude bisection, extraction
 * of S1 = Tree(X) or S2 = Tree(TS(X)) with X = supp(x*) u I, (a,b)
 * classification, canonical form and hash dedupe of the trapping sets.
 * Asynchronous: returns once the work is enqueued; the results stay in
 * device memory until ts_list_view() (which synchronizes) copies them out.
 * Errors: TSX_EINVAL (parameters), TSX_EUNSUPPORTED (decoder/degree
 * combination), TSX_ENOMEM, TSX_ECUDA.  Device-side overflows and timed-out
 * waits are reported by ts_list_view(). */
TSX_API int enumerate_ts(tsx_code *code, const tsx_enum_params *params, void *stream,
                 tsx_ts_list **out);

typedef struct {
    int64_t n_cand;        /* candidates decoded */
    int64_t n_cand_total;  /* canonical candidates of the code and rule */
    int64_t n_ts;          /* distinct trapping sets */
    int64_t decodes;
    int64_t iterations;    /* sum over decodes of the iterations executed */
    int64_t edge_updates;  /* sum over decodes of E * iterations executed */
    int64_t acyclic;       /* failing candidates with S1 = S2 = empty */
    double ms_total;       /* device time of the whole pipeline (CUDA events on the stream) */
    double ms_candidates;  /* candidate generation */
    double ms_decode;      /* the impulse-decoding kernel */
    double ms_sieve;       /* extraction, classification, canonical form and dedupe (list mode: the
                              second stage -- its decodes, sieves and inserts) */
    int64_t converged;     /* decodes that ended in the all-zero word */
    int64_t converged_iterations; /* their iterations */
    int64_t list_kstart;   /* list mode: the first iteration of the lists (0 otherwise) */
    int64_t list_patterns; /* list mode: distinct x_k sieved (consecutive equal x_k are sieved once) */
    int64_t list_iterations; /* list mode: iterations of the second stage's decodes */
} tsx_enum_stats;

/* Host views of the results, sorted by (a, b, key); valid until
 * free_ts_list().  Per trapping set i: a[i], b[i]; orbit[i] = Z / |stabilizer|
 * (1 for CSR codes); count[i] = candidates that produced it; thr[i] /
 * thr_f[i] = smallest threshold amplitude among them (min-sum integer A /
 * sum-product eps; the other is -1); flags[i] bit 0 = elementary (every
 * check touches it at most twice), bit 1 = some candidate reached it as
 * Tree(X), bit 2 = some candidate reached it as Tree(TS(X)); key: vars[var_off[i] .. var_off[i] + a[i]) ascending
 * (the lexicographically smallest circulant shift).
 * Per candidate c (if records were kept): cand_vars[4c..4c+3] canonical
 * impulse set (-1 padded); cand_thr[c] / cand_thr_f[c] threshold or -1;
 * cand_ts[c] index into the sorted list or -1; cand_flags[c] bits 0-1 =
 * sieve (0 = no failure or acyclic), bit 2 = acyclic failure, bit 3 =
 * key-pool overflow; cand_decodes[c], cand_iters[c] = decodes run and
 * iterations executed over them. */
typedef struct {
    tsx_enum_stats stats;
    int64_t n_ts;
    const int32_t *a, *b, *orbit, *count, *thr, *flags;
    const float *thr_f;
    const int64_t *var_off;
    const int32_t *vars;
    int64_t n_cand;
    const int32_t *cand_vars, *cand_thr, *cand_ts, *cand_flags, *cand_decodes, *cand_iters;
    const float *cand_thr_f;
} tsx_ts_view;

/* Synchronizes the list's stream, copies the results to host memory (once)
 * and fills `view`.  Errors: TSX_ENOMEM (the device key pool or hash table
 * overflowed), TSX_ETIMEDOUT (a device-side wait gave up), TSX_ECUDA. */
TSX_API int ts_list_view(tsx_ts_list *list, tsx_ts_view *view);

/* Device-side counters only (decodes, iterations, edge updates, number of
 * trapping sets): synchronizes and copies a few words. */
TSX_API int ts_list_stats(tsx_ts_list *list, tsx_enum_stats *stats);

TSX_API void free_ts_list(tsx_ts_list *list);

/* ---- tile autotuner (no counterpart in the paper) ---------------------
 * Picks the decode tile for `code` under `params`: the number of warps that
 * share one pair of codewords (the automatic shape -- as many pairs as fit a
 * CTA, the warps shared among them, reported as 0 -- or 1, 2, 4 or 8, at most
 * one warp per 32 rows of the smallest pass) and, for the int16 min-sum
 * decoder with sat <= 169, int8
 * message storage (which gives the same results).  Each choice decodes the
 * first num_sms * 256 canonical candidates once after one warm-up run, timed
 * with CUDA events on `stream` (synchronizes); the fastest is written to
 * `tuned` (a copy of params with decoder and warps_per_cta set) and its decode
 * time to *ms_best (may be NULL).  Float decoder and kernel = 1: tuned =
 * params.  Errors as for enumerate_ts(). */
TSX_API int tune_tile(tsx_code *code, const tsx_enum_params *params, void *stream, tsx_enum_params *tuned,
                      float *ms_best);

/* ---- batches of codes (no counterpart in the paper) -------------------
 * Enumerates several codes together: the candidate generation and the
 * sieve run per code, the impulse decodes of all codes run in ONE
 * persistent launch whose CTAs take the codes in turn and drain each
 * code's candidate queue (codes of uneven sizes share the SMs).  A batch is
 * created once (all device memory is allocated and sized there) and run any
 * number of times; batch_run() enqueues only kernels and memsets, so it can
 * be captured in a CUDA graph and replayed.
 *   codes, params: host arrays of n; every code must be on the current
 *     device; params[i].kernel = 1 (one codeword per group) and codes whose
 *     min-sum parameters leave the two-codeword kernel's 16-bit bounds, the
 *     float decoder, or a mix of QC and CSR codes or of decoders, fall back to
 *     one decode launch per code (batch_multi_launch() returns 0); a code
 *     whose two-codeword layout does not fit a CTA's shared memory gets a
 *     decode launch of its own after the multi-code one (the same kernel
 *     choice as enumerate_ts() makes for it).  At most 64 codes share the
 *     multi-code launch (more: one launch per code).
 * Results of run k are read with batch_view(batch, i, ...) after the stream
 * has reached the end of that run; batch_view synchronizes `stream` of the
 * last batch_run.  Errors as for enumerate_ts(). */
typedef struct tsx_batch tsx_batch;
TSX_API int batch_create(tsx_code *const *codes, const tsx_enum_params *params, int32_t n, void *stream,
                         tsx_batch **out);
TSX_API int batch_run(tsx_batch *batch, void *stream);
TSX_API int batch_size(const tsx_batch *batch);
TSX_API int batch_multi_launch(const tsx_batch *batch);
/* Decode launches of one batch_run(): 1 + the codes with a launch of their
 * own when the multi-code launch is used, else one per code. */
TSX_API int batch_decode_launches(const tsx_batch *batch);
/* Results of code i of the last run (same contents as ts_list_view()). */
TSX_API int batch_view(tsx_batch *batch, int32_t i, tsx_ts_view *view);
/* Sums of the device counters of all codes of the last run. */
TSX_API int batch_stats(tsx_batch *batch, tsx_enum_stats *total);
TSX_API void batch_free(tsx_batch *batch);

/* ---- importance-sampling FER toward a trapping set ------------------ */
/* The weighting step the paper takes from Cole (Sec. II-III: trapping sets
 * are weighed by importance sampling and summed into a generalized union
 * bound; the paper gives no formula).  Definition used: BPSK over AWGN with
 * sigma^2 = 1 / (2 R Eb/N0); the noise on the trapping-set bits is shifted
 * by -mu; every sample is decoded by the fixed-point min-sum decoder from
 * the all-zero codeword; FER = mean(fail * w) with
 *   log w = sum_{v in T, ascending} (n_v mu / sigma^2 - mu^2 / (2 sigma^2))
 * in double precision (mu = 0 is plain Monte Carlo).  Noise: Philox4x32-10
 * with key (job_key) and counter (v / 4, sample low, sample high, 0), four
 * uniforms u = (2 (x >> 9) + 1) 2^-24 per call, two single-precision
 * Box-Muller pairs from IEEE-rounded series; channel LLR quantized to
 * round-half-away(8 * 2 y / sigma^2), saturated to +-sat. */
typedef struct {
    double ebn0_db;        /* Eb/N0 in dB */
    double rate;           /* code rate R; 0 = 1 - m/n */
    double mu;             /* mean shift of the noise on the set's bits */
    int64_t n_samples;
    uint64_t job_key;      /* Philox key */
    int64_t sample_begin;  /* index of the first sample (for sharding) */
    int32_t K, sat, alpha_num, alpha_shift;  /* the min-sum decoder */
} tsx_is_params;

typedef struct {
    double fer;            /* mean(fail * w) */
    double var;            /* variance of that mean: (mean(w^2 fail) - fer^2) / N */
    double sum_w, sum_w2;  /* sums of fail * w and (fail * w)^2 (fixed-order reduction) */
    int64_t n_samples, n_fail;
    int64_t decodes, iterations, edge_updates;
    double ms;             /* device time (CUDA events) */
} tsx_is_result;

/* Defaults: 4 dB, R = 1 - m/n, mu = 1, 100000 samples, key 0, K = 20,
 * sat 511, alpha 3/4. */
TSX_API void is_params_default(tsx_is_params *p);

/* Runs n_samples samples on `stream` and waits for them.  ts_vars: host,
 * the a variable nodes of the trapping set (any order; duplicates ignored).
 * fail_out (host, n_samples bytes) and logw_out (host, n_samples doubles)
 * receive the per-sample failure flags and log-weights when not NULL.
 * Errors: TSX_EINVAL (node outside the code, bad parameters),
 * TSX_EUNSUPPORTED (degrees or saturation outside the decoder's 16-bit
 * bounds), TSX_ENOMEM, TSX_ECUDA. */
TSX_API int is_fer_estimate(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *params,
                            void *stream, tsx_is_result *out, uint8_t *fail_out, double *logw_out);

/* ---- the simulation decoder (Sec. III, the FER curves of Fig. 2) -------
 * Quantized normalized layered min-sum: LLR, check-to-variable and
 * variable-to-check widths of 4, 4 and 6 bits, 20 iterations.  Readings (the
 * paper names the widths only): a w-bit value saturates to
 * +-(2^(w-1) - 1); a layer is a row block of the QC base matrix; the
 * posterior P_v starts at the saturated channel value and stays at the
 * variable-to-check width; per layer and check q = sat_v2c(P_v - r),
 * r = sign * sat_c2v((alpha_num m) >> alpha_shift) with m the smallest |q| of
 * the other edges (sgn 0 = +1; a check of degree 1 sends sat_c2v), then
 * P_v = sat_v2c(q + r); x = [P < 0] and the syndrome are checked before the
 * first iteration and after each.  Failure: x != 0.  QC codes only
 * (TSX_EUNSUPPORTED otherwise). */
typedef struct {
    int32_t K;                              /* iterations (20) */
    int32_t llr_bits, c2v_bits, v2c_bits;   /* 4, 4, 6 (each 2..8) */
    int32_t alpha_num, alpha_shift;         /* 3, 2 */
} tsx_lnms_params;
TSX_API void lnms_params_default(tsx_lnms_params *p);

/* Decodes n_frames frames of channel values.  All pointers are device
 * memory: llr [n_frames][n] int8 (saturated to the LLR width here), fail
 * [n_frames] bytes out (1 = x != 0), iters [n_frames] out (may be NULL), x
 * [n_frames][n] bytes out (the decision, may be NULL).  Enqueued on `stream`,
 * not waited for.  Errors: TSX_EINVAL, TSX_EUNSUPPORTED, TSX_ENOMEM,
 * TSX_ECUDA. */
TSX_API int lnms_decode(tsx_code *code, const tsx_lnms_params *p, const int8_t *llr, int64_t n_frames,
                        uint8_t *fail, int32_t *iters, uint8_t *x, void *stream);

/* Frame-error simulation with that decoder, the way the paper's curves were
 * made (until a number of frame errors): BPSK of the all-zero word over
 * AWGN, sigma^2 = 1 / (2 R Eb/N0); the noise of frame f is the
 * importance-sampling generator's with key job_key and sample
 * frame_begin + f (mu = 0); channel value round-half-away(2 y / sigma^2 *
 * llr_scale) saturated to the LLR width.  Frames are decoded in chunks and
 * counted in order: the run stops at the first frame count whose errors
 * reach max_errors (0 = every frame), or at max_frames.  fail_out: host,
 * max_frames bytes or NULL.  Synchronizes `stream`.  Errors as for
 * lnms_decode(). */
typedef struct {
    double ebn0_db;
    double rate;        /* 0 = 1 - m/n */
    double llr_scale;   /* LLR quantization step is 1 / llr_scale (1.0) */
    int64_t max_frames;
    int64_t max_errors; /* 200 */
    uint64_t job_key;
    int64_t frame_begin;
} tsx_sim_params;
typedef struct {
    int64_t frames, frame_errors, bit_errors;
    double fer, ber;    /* frame_errors / frames, bit_errors / (frames n) */
    int64_t iterations, edge_updates;
    double ms;          /* device time of the decode launches (CUDA events) */
} tsx_sim_result;
TSX_API void sim_params_default(tsx_sim_params *p);
TSX_API int lnms_simulate(tsx_code *code, const tsx_lnms_params *p, const tsx_sim_params *sp, void *stream,
                          tsx_sim_result *out, uint8_t *fail_out);

/* ---- the generalized union bound (Sec. II-III) --------------------------
 * The error-floor estimate the paper builds from the trapping-set list with
 * Cole's weighting: FER_UB = sum over the sets of mult_i * FER_i, FER_i the
 * importance-sampling estimate of is_fer_estimate() toward set i with job key
 * params->job_key + i, and its variance sum mult_i^2 var_i.  ts_vars: host,
 * the sets' variable nodes one after the other, set i at
 * ts_vars[ts_off[i] .. ts_off[i+1]); mult: host, n_sets multiplicities (the
 * orbit sizes of a QC list, 1 for a general code); fer_out: host, n_sets
 * per-set estimates or NULL.  The sets' sampling launches are enqueued on
 * `stream` together and waited for once.  Errors as for is_fer_estimate(). */
typedef struct {
    double fer_ub, var_ub;
    int64_t n_sets, samples, n_fail, edge_updates;
    double ms;          /* device time from the first launch to the last (CUDA events) */
} tsx_union_result;
TSX_API int union_bound_fer(tsx_code *code, int64_t n_sets, const int32_t *ts_vars, const int64_t *ts_off,
                            const double *mult, const tsx_is_params *params, void *stream, tsx_union_result *out,
                            double *fer_out);

/* ---- serving runtime (no counterpart in the paper) --------------------
 * A request loop over resident codes: enumeration and importance-sampling
 * jobs are submitted as they arrive, admitted in arrival order while their
 * device-memory footprint fits the server's budget and a job slot is free
 * (a job that does not fit may be overtaken by later ones that do, for at
 * most backfill_ms), and run concurrently on a pool of streams: each job's
 * persistent launches are sized to its work and split into chunks, so that
 * jobs arriving while others are on the GPU get SMs at the next chunk
 * boundary; small jobs run on high-priority streams, large ones on
 * low-priority streams, at most max_large of them at once.  A job's results
 * are the same as those of the stand-alone entry point with the same
 * parameters (chunking and grid size do not change them).  One host thread
 * of the server drives the GPU; the calls below may come from any thread. */
typedef struct tsx_server tsx_server;

enum { TSX_JOB_ENUMERATE = 0, TSX_JOB_IS_FER = 1 };

typedef struct {
    int32_t max_jobs;          /* jobs on the device at once (default 8) */
    int32_t serial;            /* 1: the plain method -- one job at a time in arrival order,
                                  each as one full-GPU launch per step (for comparison) */
    int32_t device;            /* CUDA device; -1 = the current one */
    int64_t hbm_bytes;         /* device memory the admitted jobs may hold together;
                                  0 = half of the free memory at creation */
    int64_t chunk_candidates;  /* decode launch granularity of enumeration jobs (default 16384) */
    int64_t chunk_samples;     /* launch granularity of IS jobs (default 32768) */
    double small_work;         /* jobs whose estimated edge updates -- candidates x (s+1)/2 x E x K/2,
                                  or samples x E x K/2 -- are at most this run on high-priority
                                  streams (default 2e10) */
    double backfill_ms;        /* how long a job that does not fit may be overtaken (default 100) */
    int32_t max_large;         /* large (low-priority) jobs on the device at once, in arrival
                                  order among themselves (default 1) */
} tsx_server_params;

typedef struct {
    int32_t kind;                  /* TSX_JOB_* */
    tsx_code *code;                /* a loaded code; keep it loaded until the job is done */
    tsx_enum_params enum_params;   /* TSX_JOB_ENUMERATE (the results are kept as by enumerate_ts) */
    tsx_is_params is_params;       /* TSX_JOB_IS_FER */
    const int32_t *ts_vars;        /* TSX_JOB_IS_FER: host, a variable nodes (copied at submit) */
    int32_t a;
} tsx_job;

typedef struct {
    int32_t status;        /* TSX_OK, TSX_EAGAIN (queued or running) or the job's error */
    int32_t kind;
    int32_t high_priority; /* ran on a high-priority stream */
    int32_t grid_sms;      /* SMs its persistent launches were sized to */
    int64_t device_bytes;  /* admitted footprint */
    double queue_ms;       /* submit -> admission */
    double run_ms;         /* admission -> results on the host */
    double latency_ms;     /* submit -> results on the host */
    tsx_enum_stats enum_stats;
    tsx_is_result is_result;
} tsx_job_result;

typedef struct {
    int64_t submitted, done, failed, running, queued;
    double p50_ms, p90_ms, p99_ms, max_ms, mean_ms;  /* latency of the completed jobs */
    double mean_queue_ms;
    double makespan_ms;        /* first submit -> last completion */
    int64_t edge_updates, decodes;
    double edge_updates_per_s; /* edge_updates / makespan */
    int64_t hbm_peak_bytes;    /* largest admitted footprint held at once */
    int32_t max_concurrent;    /* most jobs on the device at once */
} tsx_server_stats;

/* Defaults as stated above (max_jobs 8, serial 0, device -1, ...). */
TSX_API void server_params_default(tsx_server_params *p);
/* Creates the server and its worker thread.  Errors: TSX_EINVAL, TSX_ECUDA. */
TSX_API int server_create(const tsx_server_params *params, tsx_server **out);
/* Queues a job and returns its id.  The parameters are validated and the
 * footprint computed here: TSX_EINVAL / TSX_EUNSUPPORTED as for the
 * stand-alone call, TSX_ENOMEM if the job alone exceeds the budget. */
TSX_API int server_submit(tsx_server *server, const tsx_job *job, uint64_t *id);
/* TSX_EAGAIN while the job is queued or running; TSX_ENOTFOUND for an
 * unknown or released id; otherwise fills `result` and returns its status. */
TSX_API int server_poll(tsx_server *server, uint64_t id, tsx_job_result *result);
/* As server_poll, but waits up to timeout_ms (< 0: without limit). */
TSX_API int server_wait(tsx_server *server, uint64_t id, double timeout_ms, tsx_job_result *result);
/* Results of a completed enumeration job (valid until server_release). */
TSX_API int server_job_view(tsx_server *server, uint64_t id, tsx_ts_view *view);
/* Forgets a completed job and its results (TSX_EAGAIN if not completed). */
TSX_API int server_release(tsx_server *server, uint64_t id);
/* Waits until every submitted job has completed. */
TSX_API int server_drain(tsx_server *server);
TSX_API int server_stats(tsx_server *server, tsx_server_stats *stats);
/* Clears the latency record and counters (jobs in flight are kept). */
TSX_API void server_reset_stats(tsx_server *server);
/* Waits for the jobs on the device, drops the queued ones, frees everything. */
TSX_API void server_destroy(tsx_server *server);

/* ---- decoding without allocation (no counterpart in the paper) --------
 * For callers that cannot allocate device memory -- a latency-critical host
 * thread that must not take the driver's allocation locks, code running
 * under another framework's memory manager that forbids outside cudaMalloc,
 * or a process that has reserved the whole device -- this entry point runs
 * the impulse decodes with amplitude bisection (the kernel enumerate_ts()
 * uses) on candidate sets the caller supplies, and keeps all of its working
 * memory in one fixed device array of TSX_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   code:      a code loaded earlier with load_code() on the current device.
 *   params:    as for enumerate_ts(); the candidate fields are ignored.
 *   cand_vars: device, 16-byte aligned, n_cand x 4 int32: variable nodes of
 *              each impulse set, -1 padded at the end (1 to 4 nodes).
 *   thr:       device, n_cand int32 out: min-sum threshold amplitude, -1 if
 *              the decoder never failed (and -1 for the float decoder).
 *   thr_f:     device, n_cand float out (may be NULL): float-decoder
 *              threshold eps, -1 otherwise.
 *   decodes, iters: device, n_cand int32 out: decodes run and iterations
 *              executed per candidate.
 * Returns TSX_ENOMEM, without touching the outputs, when
 *   n_cand * (28 + 4 * ceil(n / 32)) + ~2 KB > TSX_NOALLOC_SCRATCH_BYTES,
 * TSX_EINVAL for a malformed candidate set (checked on the device; this
 * check waits for the stream), a misaligned pointer or a code loaded on
 * another device.  The call waits for `stream` once, after the candidate
 * check; the decode itself is enqueued on `stream` and not waited for.  The
 * first call on each device looks up the array's device address (make that
 * first call before any stream capture).  Every call uses the
 * same array and finds the previous call's contents in it; the counters it
 * relies on are reset at the start of each call, so calls that overlap on
 * the GPU (on different streams or threads) race and must not be issued. */
#define TSX_NOALLOC_SCRATCH_BYTES (16u << 20)
TSX_API int decode_thresholds_noalloc(const tsx_code *code, const tsx_enum_params *params,
                                      const int32_t *cand_vars, int64_t n_cand, int32_t *thr, float *thr_f,
                                      int32_t *decodes, int32_t *iters, void *stream);

/* ---- measured issue rates (no counterpart in the paper) ----------------
 * The decoders are bound by integer issue and shared-memory bandwidth, for
 * which no vendor figure is measured on the part.  measure_peaks() runs one
 * short probe kernel per quantity with every SM full and reads each SM's
 * cycle counter around its CTAs: the result is per SM clock (independent of
 * the clock the GPU ran at), the median over SMs.  Multiply by the SM count
 * and an SM clock to get a peak.  Synchronizes `stream`; allocates and frees
 * a few KB of device memory.  Errors: TSX_EINVAL, TSX_ENOMEM, TSX_ECUDA. */
typedef struct {
    int32_t num_sms;               /* multiprocessors of the current device */
    double int32_ops_per_clk_sm;   /* 32-bit integer lane operations (min.u32, xor) */
    double u16x2_ops_per_clk_sm;   /* packed 16-bit lane operations (min.u16x2, xor): each serves two values */
    double smem_bytes_per_clk_sm;  /* shared-memory load bytes (16-byte vector loads, no bank conflict) */
    double sfu_ops_per_clk_sm;     /* special-function lane operations (ex2.approx.f32) */
    double fp32_fma_per_clk_sm;    /* single-precision fused multiply-add lane operations */
    double imad_ops_per_clk_sm;    /* 32-bit integer multiply-add lane operations (mad.lo.u32) */
} tsx_peaks;
TSX_API int measure_peaks(tsx_peaks *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TSX_H */
