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

// Computes the slot layout for a decoder and picks a shape: G warps per
// codeword (0 = automatic) and groups per CTA (0 = automatic); ctas_per_sm
// 0 = as many as fit.  Returns false if one codeword does not fit.
bool plan_shape(const DevCode &g, int decoder, int G, int groups, int ctas_per_sm, int num_sms,
                LaunchShape *out);

cudaError_t launch_enum(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                        const LaunchShape &sh, cudaStream_t st);

// Compacts the hash table: assigns each stored trapping set an index,
// writes its pool offset / count / min threshold, and rewrites the
// candidates' slots as indices.
cudaError_t launch_compact(const EnumBuffers &b, long long n_rec, int *ts_off, int *ts_count,
                           int *ts_thr, int *slot_map, cudaStream_t st);

}  // namespace tsx
