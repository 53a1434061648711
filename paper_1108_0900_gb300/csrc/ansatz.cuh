// Parameter loads and correlator state arithmetic of the CPS x pfaffian
// ansatz (Eq. 11) shared by the walker kernels and the linear-method product.
#pragma once
#include "common.cuh"

namespace vmc {

template <typename R>
__device__ __forceinline__ R load_F(const DevProblem& pb, int p, int q);
template <> __device__ __forceinline__ float load_F<float>(const DevProblem& pb, int p, int q) {
    return __ldg(pb.F32 + p * pb.M + q);
}
template <> __device__ __forceinline__ double load_F<double>(const DevProblem& pb, int p, int q) {
    return __ldg(pb.F64 + p * pb.M + q);
}
template <typename R> __device__ __forceinline__ R load_C(const DevProblem& pb, int64_t k);
template <> __device__ __forceinline__ float load_C<float>(const DevProblem& pb, int64_t k) {
    return __ldg(pb.C32 + k);
}
template <> __device__ __forceinline__ double load_C<double>(const DevProblem& pb, int64_t k) {
    return __ldg(pb.C64 + k);
}

// weight 4^j of site s inside correlator c (0 if absent): one table load
__device__ __forceinline__ int site_weight_in(const DevProblem& pb, int c, int s) {
    return (int)__ldg(pb.corr_site_w + c * pb.ns + s);
}

// Correlator part of Psi(n')/Psi(n) for moving one electron of spin factor
// sf (1 up, 2 down) from site sp to site sq.  Entry e of the concatenated
// membership lists of sp and sq; a correlator holding both sites is handled
// once (from sp's list).  Returns the factor and the new state in *newidx
// (or -1 when the entry contributes nothing).
__device__ __forceinline__ int corr_entry(const DevProblem& pb, const uint32_t* cidx, int sp, int sq,
                                          int sf, int e, int* cout) {
    int dp = pb.site_cptr[sp + 1] - pb.site_cptr[sp];
    if (e < dp) {
        int ent = pb.site_cptr[sp] + e;
        int c = pb.site_corr[ent];
        int newi = (int)cidx[c] - sf * pb.site_w[ent] + sf * site_weight_in(pb, c, sq);
        *cout = c;
        return newi;
    }
    int ent = pb.site_cptr[sq] + (e - dp);
    int c = pb.site_corr[ent];
    if (site_weight_in(pb, c, sp) != 0) { *cout = -1; return -1; }
    *cout = c;
    return (int)cidx[c] + sf * pb.site_w[ent];
}

}  // namespace vmc
