// tsx_internal.cuh -- device-side data layout shared by the library's kernels.
//
// Layout in HBM (per loaded code, resident until free_code):
//   QC codes keep only the exponent matrix in derived per-row-block and
//   per-column-block tables (a few hundred bytes); every neighbour index is
//   computed from a shift, never stored per edge.  General (CSR) codes keep
//   uint16 adjacency arrays.  Both keep the Tanner balls of the orbit
//   representatives (sorted int32 lists).
// Edge numbering (the message layout in shared memory):
//   QC:  check (i, r), position p (p-th non-zero block of row block i, in
//        ascending column order) -> e = reoff[i] + p*Z + r, so consecutive
//        lanes (consecutive r) touch consecutive messages.
//   CSR: check-major, e = c_ptr[c] + p.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsx.h"

namespace tsx {

constexpr int kMaxDc = TSX_MAX_DC;
constexpr int kMaxDv = TSX_MAX_DV;
constexpr int kMaxNb = TSX_MAX_NB;
constexpr int kMaxMb = 64;

struct DevCode {
    int kind;  // TSX_CODE_QC / TSX_CODE_CSR
    int n, m, E, Z, n_b, m_b;
    int dv_max, dc_max;
    int dc_min;         // smallest check degree (dc_min == dc_max: check-regular)
    int dv_min;         // smallest variable degree (dv_min == dv_max: variable-regular)
    int girth, wstart;  // wstart = max(1, girth/2)
    int n_rep;
    // QC tables
    const int16_t *rdeg;   // [m_b]
    const int32_t *reoff;  // [m_b]
    const int32_t *rjz;    // [m_b * dc_max]  (column block j of position p) * Z
    const int16_t *rs;     // [m_b * dc_max]  its shift
    const int16_t *cdeg;   // [n_b]
    const int32_t *ceoff;  // [n_b * dv_max]  reoff[i] + p*Z of the t-th block of column j
    const int16_t *cs;     // [n_b * dv_max]  its shift
    const int32_t *ciz;    // [n_b * dv_max]  its row block i * Z
    // CSR tables (uint16; E < 65536)
    const uint16_t *c_ptr;   // [m+1]
    const uint16_t *c_vn;    // [E]
    const uint16_t *v_ptr;   // [n+1]
    const uint16_t *v_edge;  // [E] edges of v, ascending check
    const uint16_t *v_chk;   // [E] check of that edge
    // Tanner balls of the representatives
    const int64_t *ball_ptr;  // [n_rep+1]
    const int32_t *ball;
};

// Device-wide counters and flags of one enumeration.
struct Counters {
    unsigned long long next_cand;   // work queue head of a single-launch decode
    unsigned long long decodes;
    unsigned long long iterations;
    unsigned long long edge_updates;
    unsigned long long pool_top;    // int32 words used in the key pool
    unsigned long long n_cand_total;  // canonical candidates written
    unsigned long long acyclic;
    unsigned long long next_sieve;  // work queue of the sieve kernel
    unsigned long long n_fail;      // importance sampling: failing samples
    unsigned long long pool_leaked; // key-pool words reserved by an insert that lost to an equal key
                                    // and could not be given back
    unsigned long long ok_decodes;  // decodes that ended in the all-zero word
    unsigned long long ok_iters;    // their iterations
    unsigned long long list_patterns;  // list mode: x_k patterns sieved
    unsigned long long list_iters;     // list mode: iterations of the second stage
    unsigned long long list_kstart;    // list mode: first iteration of the lists
    unsigned int n_ts;
    unsigned int err;               // bit flags, see kErr*
};

constexpr unsigned kErrPoolOverflow = 1u;
constexpr unsigned kErrTableFull = 2u;
constexpr unsigned kErrCandOverflow = 4u;
constexpr unsigned kErrCycleOverflow = 8u;

// Per-candidate flags
constexpr int kFlagSieveMask = 3;
constexpr int kFlagAcyclic = 4;
constexpr int kFlagOverflow = 8;

// Per-TS record header in the key pool: [a, b, orbit, flags, key...]
constexpr int kPoolHdr = 4;

struct DecodeParams {
    int decoder;  // TSX_DEC_*
    int K;
    int base_llr;
    int sat;
    int alpha_num, alpha_shift;
    int amp_steps;
    float spa_clip, spa_amax;
};

struct EnumBuffers {
    const int4 *cands;        // canonical candidate sets, -1 padded
    long long cand_begin;     // first candidate to decode
    long long cand_end;       // one past the last (clamped to the total on device)
    int record;               // (unused on the device: records are always kept)
    // decode work queue: the next candidate is cand_begin + atomicAdd(*queue, 1);
    // records are indexed by (candidate - rec_base).  A list decoded in one
    // launch has queue = &ctr->next_cand and rec_base = cand_begin; a list
    // decoded in chunks gives every chunk launch its own queue word and range.
    unsigned long long *queue;
    long long rec_base;
    // per-candidate outputs, indexed by (candidate - rec_base)
    int *c_thr;
    float *c_thr_f;
    int *c_slot;
    int *c_flags;
    int *c_decodes;
    int *c_iters;
    // per-candidate iteration limits (indexed like cands), or null: every
    // candidate gets K (the cycle-density budgets of budget_kernel)
    const uint16_t *cand_K;
    // best error pattern x* of every failing candidate, nw words each
    uint32_t *xstar;
    int nw;
    // trapping-set hash table
    unsigned long long *tags;  // [cap] (hash_hi32 << 32) | pool offset, 0 = empty
    int *t_thr;                // [cap] min threshold, int-ordered
    int *t_count;              // [cap]
    unsigned long long cap_mask;
    int *pool;
    unsigned long long pool_cap;
    Counters *ctr;
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrapZ(int x, int Z) {
    // x in [0, 2Z) -> x mod Z
    return (unsigned)x < (unsigned)Z ? x : x - Z;
}
__device__ __forceinline__ int wrapZneg(int x, int Z) {
    // x in [-Z, Z) -> x mod Z
    return x < 0 ? x + Z : x;
}
__device__ __forceinline__ int clampi(int x, int lo, int hi) { return min(max(x, lo), hi); }
__device__ __forceinline__ float clampf_(float x, float lo, float hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // SplitMix64 finalizer (Steele, Lea, Flood 2014)
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Float thresholds are stored in the int-ordered min table: for non-negative
// floats the IEEE bit pattern orders like the value.
__device__ __forceinline__ int f2ord(float f) { return __float_as_int(f); }

}  // namespace tsx
