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

}  // namespace tsx
