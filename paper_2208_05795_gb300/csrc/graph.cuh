// graph.cuh -- neighbour access on the device tables of a loaded code.
//
// QC (eqs. 1-2): variable node (j,k) sits in check (i, (k - a_ij) mod Z) of
// every row block i with a_ij >= 0; check (i,r) holds variable node
// (j, (r + a_ij) mod Z) of every column block j with a_ij >= 0.
#pragma once
#include "tsx_internal.cuh"

namespace tsx {

// Degree of variable node v / check c.
__device__ __forceinline__ int vn_degree(const DevCode &g, int v) {
    if (g.kind == TSX_CODE_QC) return g.cdeg[v / g.Z];
    return g.v_ptr[v + 1] - g.v_ptr[v];
}
__device__ __forceinline__ int cn_degree(const DevCode &g, int c) {
    if (g.kind == TSX_CODE_QC) return g.rdeg[c / g.Z];
    return g.c_ptr[c + 1] - g.c_ptr[c];
}
// t-th check of v (ascending)
__device__ __forceinline__ int vn_check(const DevCode &g, int v, int t) {
    if (g.kind == TSX_CODE_QC) {
        int j = v / g.Z, k = v - j * g.Z;
        int idx = j * g.dv_max + t;
        return g.ciz[idx] + wrapZneg(k - g.cs[idx], g.Z);
    }
    return g.v_chk[g.v_ptr[v] + t];
}
// p-th variable node of c (ascending)
__device__ __forceinline__ int cn_vn(const DevCode &g, int c, int p) {
    if (g.kind == TSX_CODE_QC) {
        int i = c / g.Z, r = c - i * g.Z;
        int idx = i * g.dc_max + p;
        return g.rjz[idx] + wrapZ(r + g.rs[idx], g.Z);
    }
    return g.c_vn[g.c_ptr[c] + p];
}
// representative variable node of orbit representative index rep
__device__ __forceinline__ int rep_vn(const DevCode &g, int rep) {
    return g.kind == TSX_CODE_QC ? rep * g.Z : rep;
}
// circulant shift of variable node v by s (QC); identity for CSR
__device__ __forceinline__ int shift_vn(const DevCode &g, int v, int s) {
    if (g.kind != TSX_CODE_QC) return v;
    int j = v / g.Z, k = v - j * g.Z;
    int kk = k + s;
    kk %= g.Z;
    if (kk < 0) kk += g.Z;
    return j * g.Z + kk;
}

}  // namespace tsx
