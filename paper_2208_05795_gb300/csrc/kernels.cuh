// kernels.cuh -- launch interfaces of the library's kernels (host side).
#pragma once
#include "tsx_internal.cuh"

namespace tsx {

// ---- candidate generation (cand.cu) -------------------------------------
struct CandArgs {
    DevCode code;
    int max_size;
    const long long *raw_off;  // [n_rep + 1] raw-set offsets per representative
    long long raw_total;
    int *chunk_count;          // [n_chunks]
    const long long *chunk_off;  // [n_chunks + 1]
    int4 *cands;
    Counters *ctr;
};

struct CycleArgs {
    DevCode code;
    int l;              // VNs per cycle
    long long paths;    // path-index space per representative
    int *count;         // [n_rep]
    const long long *off;  // [n_rep + 1] (absolute positions in cands)
    int4 *cands;
    Counters *ctr;
};

cudaError_t launch_ball(const DevCode &g, int *sizes, const int64_t *ptr, int32_t *ball, bool write,
                        cudaStream_t st);
cudaError_t launch_cand_ball(const CandArgs &a, long long n_chunks, bool write, cudaStream_t st);
cudaError_t launch_cand_cycle(const CycleArgs &a, bool write, cudaStream_t st);
// Exclusive scan of n counts into off[0..n], starting at *base (0 if
// null); with add_total the grand total becomes the candidate count.
cudaError_t launch_scan(const int *cnt, long long n, long long *off, const long long *base, Counters *ctr,
                        bool add_total, cudaStream_t st);
long long cand_chunks(long long raw_total);
// Per-candidate iteration limits of the cycle-density budget for the first
// min(bound, candidate count) candidates.
cudaError_t launch_budget(const int4 *cands, long long bound, const int *vweight, int K, int kmin, int wref,
                          uint16_t *cand_K, const Counters *ctr, cudaStream_t st);

// ---- impulse decoding, bisection, extraction, dedupe (decode.cu) --------
struct SlotLayout {
    int tables_bytes;  // shared code tables at the start of the CTA's shared memory
    int r_off, p_off, xa_off, xb_off, misc_off;  // offsets inside a slot
    int slot_bytes;
};

struct LaunchShape {
    int G;           // warps per codeword group
    int groups;      // groups per CTA
    int ctas;        // grid size (persistent), recomputed from the occupancy at launch
    int num_sms;
    int per_sm_req;  // requested CTAs per SM (0 = as many as are resident)
    int smem_bytes;  // dynamic shared memory per CTA
    SlotLayout lay;
};

// One code of a multi-code decode launch.
struct BatchItem {
    DevCode g;
    DecodeParams dp;
    EnumBuffers b;
    SlotLayout lay;
    int G, groups;
    int scalar;  // 1: not in the multi-code launch (its pair layout does not fit a CTA)
};

// All items of a multi-code launch, passed by value as one kernel parameter
// (kernel parameters may take up to 32 KB).
constexpr int kMaxBatch = 64;

// warps per CTA of the single-code two-codeword kernel (its launch bound):
// 20 warps keep the (3,6)-regular general-code variant at 96 registers
// without spills and measured faster than 16 or 24
constexpr int kPairWarps = 20;
// QC codes and general codes of check degree 7 or 8: 16 warps a CTA (128
// registers a thread, which those variants need to run without spilling)
constexpr int kPairWarps16 = 16;
__host__ __device__ constexpr int pair_kernel_warps(bool qc, int dc, bool exact) {
    return qc || (dc == 8 && !exact) ? kPairWarps16 : kPairWarps;
}
// warps per CTA of the importance-sampling kernel's flat form (its launch bound)
constexpr int kIsWarps = 18;
struct BatchArgs {
    BatchItem it[kMaxBatch];
};
static_assert(sizeof(BatchArgs) + 64 <= 32764, "batch kernel parameters above 32 KB");

// Plans a multi-code launch of the two-codewords-per-lane kernel (fills
// items[] on the host and the common shape over the items that take part);
// a code whose pair layout does not fit a CTA's shared memory gets
// scalar = 1 and is left to a launch of its own.  False if the codes cannot
// share one kernel (kind, decoder or 16-bit bounds differ).
bool plan_batch(const DevCode *const *g, const DecodeParams *dp, const EnumBuffers *b, const int *G_req, int n,
                int num_sms, BatchItem *items, LaunchShape *common, int *variant);
// Launches it over the device copy of items[].
cudaError_t launch_batch(const BatchArgs &items, int n, int variant, const LaunchShape &sh, cudaStream_t st);

// Runs the impulse decodes with bisection over the candidates of b and
// writes the per-candidate records and x* of failing candidates.  NMS
// decoders use the two-codeword kernel where its 16-bit bias bounds hold
// (else, or with force_scalar, the one-codeword kernel).  G / groups /
// ctas_per_sm: 0 = automatic.
cudaError_t launch_decode(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, int G, int groups,
                          int ctas_per_sm, int num_sms, int force_scalar, cudaStream_t st);

// Sieve (Tree / TS), classification, canonical key and hash insert of every
// failing candidate (reads the records and x* written by the decoder).
cudaError_t launch_sieve(const DevCode &g, const EnumBuffers &b, int decoder, int num_sms, cudaStream_t st);

// Shape of the importance-sampling kernel (two samples per lane); false if
// the 16-bit bias bounds or the shared memory do not allow it.
bool plan_is_shape(const DevCode &g, const DecodeParams &dp, LaunchShape *sh, int num_sms);

// Whether one codeword of g fits the shared memory of a CTA.
bool decode_fits(const DevCode &g, int decoder);

// ---- the ordered list of Sec. III (list.cu) --------------------------------
// Whether one group's list-mode slot fits a CTA for iteration limit K.
bool list_fits(const DevCode &g, int K);
// The second stage over the failing candidates of b (after the decode):
// replay at the threshold, sieve every x_k from kstart (0: floor(girth/2),
// -1: ceil of the first stage's average converged iterations), insert.
cudaError_t launch_list(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, int kstart, int num_sms,
                        cudaStream_t st);

// ---- short cycles (cycles.cu) ------------------------------------------------
constexpr int kCycLmax = 6;     // variable nodes per cycle at most
constexpr int kEmdBins = 128;   // EMD values per length
// Closed walks from the representatives, per representative and number of
// variable nodes (walks[n_rep][kCycLmax + 1]) and, with hist, per number of
// variable nodes and EMD (hist[kCycLmax + 1][kEmdBins]); zeroed first.
cudaError_t launch_cycles(const DevCode &g, int lmax, unsigned long long *walks, unsigned long long *hist,
                          cudaStream_t st);

// accessors of a loaded code (api.cu)
const DevCode *code_dev(const tsx_code *c);
int code_num_sms(const tsx_code *c);
int code_device(const tsx_code *c);
// validates enumeration parameters and extracts the decoder's part
int enum_params_to_decode(const tsx_enum_params *p, DecodeParams *dp);

// Compacts the hash table: assigns each stored trapping set an index,
// writes its pool offset / count / min threshold, and rewrites the
// candidates' slots as indices.
cudaError_t launch_compact(const EnumBuffers &b, long long n_rec, int *ts_off, int *ts_count,
                           int *ts_thr, int *slot_map, cudaStream_t st);

// ---- serving runtime hooks ------------------------------------------------
// enumeration lists (api.cu): device bytes and candidate bound of a list, start (allocate and
// enqueue everything), finish (after the stream passed: results to the host,
// device memory back), delete.  dchunk > 0 splits the decode into launches of
// dchunk candidates; grid_sms > 0 caps the persistent grids at that many SMs.
int list_bytes(tsx_code *code, const tsx_enum_params *params, long long dchunk, long long *bytes,
               long long *cand_bound);
int list_start(tsx_code *code, const tsx_enum_params *params, cudaStream_t s, long long dchunk, int grid_sms,
               tsx_ts_list **out);
long long list_cand_bound(const tsx_ts_list *L);
int list_finish(tsx_ts_list *L);
void list_delete(tsx_ts_list *L);

// importance-sampling jobs (isfer.cu), the same protocol; chunk > 0 splits
// the samples into launches of chunk samples (results do not change).
struct IsJob;
int is_job_bytes(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p, long long chunk,
                 long long *bytes);
int is_job_start(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p, cudaStream_t s,
                 long long chunk, int grid_sms, IsJob **out);
int is_job_finish(IsJob *J, tsx_is_result *out, uint8_t *fail_out, double *logw_out);
void is_job_delete(IsJob *J);

}  // namespace tsx
