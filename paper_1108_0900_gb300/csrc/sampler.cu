// Walker kernels: Metropolis sampling from |Psi_n|^2 (Sec. II.A, fixed N and
// S_z as in Sec. III), local energy, and the per-sample derivative ratios
// O_k(n) = Psi^k_n / Psi_n of Eq. 3 for the CPS x pfaffian ansatz of Eq. 11.
//
// One warp owns one walker.  The walker keeps X = A^{-1}, A = F[occ, occ],
// in shared memory with the electron positions left unsorted (a move puts
// the new orbital in the vacated position).  For a move p -> q at position a
// with b_j = F[q, o_j] (b_a = 0):
//   Pf(A')/Pf(A) = sum_j b_j X_{ja} = -sum_j b_j X_{aj}
// (Pf is linear in row/column a; dPf/dA_aj = Pf X_{ja}).  The Jordan-Wigner
// sign of the hop cancels the sign of re-sorting the positions, so this
// unsorted ratio is the signed amplitude ratio the local energy needs.  On
// acceptance A' = A + e_a u^T - u e_a^T (u = b - A_{a,:}), whose 2x2
// Woodbury capacitance is r I, so
//   X' = X + (c y^T - y c^T) / r,  c = X_{:,a},  y = X b + e_a.
// The inverse is rebuilt from scratch (Gauss-Jordan, partial pivoting) at
// the start of every call.  The chain also sums ln|ratio| of its accepted
// moves (the logarithm in the chain's precision, the sum in FP64), the
// running log-amplitude that a from-scratch evaluation of the stored samples
// checks (vmc_sample_stats).
#include "ansatz.cuh"
#include "common.cuh"
#include "kernels.h"

namespace vmc {

struct WarpMem {
    unsigned char* base;
};


// ln|x| in the walker's precision (FP32 chains avoid the FP64 pipe)
__device__ __forceinline__ float log_abs(float x) { return logf(fabsf(x)); }
__device__ __forceinline__ double log_abs(double x) { return log(fabs(x)); }

// Sum of many terms of the walker's precision with FP64 accuracy: FP64 for
// FP64 walkers; for FP32 walkers an FP32 pair (two-sum: the rounding error of
// each add goes to the low word), which keeps the sum off the FP64 pipe.
template <typename R> struct term_sum;
template <> struct term_sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct term_sum<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x);
        const float bx = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bx)), __fsub_rn(x, bx)));
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename R> struct pair_of;
template <> struct pair_of<float> { using type = float2; };
template <> struct pair_of<double> { using type = double2; };

template <typename R>
__device__ R corr_ratio_warp(const DevProblem& pb, uint32_t* cidx, int p, int q, bool commit) {
    const int lane = threadIdx.x & 31;
    int ns = pb.ns;
    int sf = p >= ns ? 2 : 1;
    int sp = p >= ns ? p - ns : p, sq = q >= ns ? q - ns : q;
    int total = (pb.site_cptr[sp + 1] - pb.site_cptr[sp]) + (pb.site_cptr[sq + 1] - pb.site_cptr[sq]);
    R prod = R(1);
    for (int base = 0; base < total; base += 32) {
        int e = base + lane;
        R r = R(1);
        int c = -1, newi = -1;
        if (e < total) {
            newi = corr_entry(pb, cidx, sp, sq, sf, e, &c);
            if (c >= 0) r = load_C<R>(pb, pb.corr_off[c] + newi) / load_C<R>(pb, pb.corr_off[c] + cidx[c]);
        }
        prod *= warp_prod(r);
        if (commit) {
            __syncwarp();
            if (c >= 0) cidx[c] = (uint32_t)newi;
            __syncwarp();
        }
    }
    return prod;
}

// lane-serial version used while every lane evaluates its own hop
template <typename R>
__device__ R corr_ratio_serial(const DevProblem& pb, const uint32_t* cidx, int p, int q) {
    int ns = pb.ns;
    int sf = p >= ns ? 2 : 1;
    int sp = p >= ns ? p - ns : p, sq = q >= ns ? q - ns : q;
    int total = (pb.site_cptr[sp + 1] - pb.site_cptr[sp]) + (pb.site_cptr[sq + 1] - pb.site_cptr[sq]);
    R prod = R(1);
#pragma unroll 4
    for (int e = 0; e < total; ++e) {
        int c;
        int newi = corr_entry(pb, cidx, sp, sq, sf, e, &c);
        if (c >= 0) prod *= load_C<R>(pb, pb.corr_off[c] + newi) / load_C<R>(pb, pb.corr_off[c] + cidx[c]);
    }
    return prod;
}

// In-place Gauss-Jordan inverse with partial pivoting of the N x N matrix X
// (row stride XS) by one warp.  col: N scratch, piv: N row indices.  Returns
// false if a pivot column is entirely zero or not finite.
template <typename R>
__device__ bool gj_invert_warp(R* X, int N, int XS, R* col, uint8_t* piv) {
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < N; ++k) {
        R best = R(-1);
        int bi = N;
        for (int i = k + lane; i < N; i += 32) {
            R v = fabs(X[i * XS + k]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            R ob = __shfl_xor_sync(VMC_FULL_MASK, best, o);
            int oi = __shfl_xor_sync(VMC_FULL_MASK, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > R(0)) || !isfinite(best)) return false;
        if (lane == 0) piv[k] = (uint8_t)bi;
        if (bi != k) {
            for (int j = lane; j < N; j += 32) {
                R t = X[k * XS + j];
                X[k * XS + j] = X[bi * XS + j];
                X[bi * XS + j] = t;
            }
        }
        __syncwarp();
        R pinv = R(1) / X[k * XS + k];
        for (int i = lane; i < N; i += 32) col[i] = X[i * XS + k];
        __syncwarp();
        for (int j = lane; j < N; j += 32) X[k * XS + j] = (j == k ? R(1) : X[k * XS + j]) * pinv;
        __syncwarp();
        for (int j = lane; j < N; j += 32) {
            R rk = X[k * XS + j];
            for (int i = 0; i < N; ++i) {
                if (i == k) continue;
                R x = (j == k) ? R(0) : X[i * XS + j];
                X[i * XS + j] = x - col[i] * rk;
            }
        }
        __syncwarp();
    }
    for (int k = N - 1; k >= 0; --k) {
        int pk = piv[k];
        if (pk != k) {
            for (int i = lane; i < N; i += 32) {
                R t = X[i * XS + k];
                X[i * XS + k] = X[i * XS + pk];
                X[i * XS + pk] = t;
            }
        }
        __syncwarp();
    }
    return true;
}

template <typename R> __device__ __forceinline__ R load_h(const DevProblem& pb, int i, int j);
template <> __device__ __forceinline__ float load_h<float>(const DevProblem& pb, int i, int j) {
    return __ldg(pb.h32 + i * pb.ns + j);
}
template <> __device__ __forceinline__ double load_h<double>(const DevProblem& pb, int i, int j) {
    return __ldg(pb.h64 + i * pb.ns + j);
}
// (pq|rs) over spatial orbitals
template <typename R> __device__ __forceinline__ R load_eri(const DevProblem& pb, int p, int q, int r, int s);
template <> __device__ __forceinline__ float load_eri<float>(const DevProblem& pb, int p, int q, int r, int s) {
    const int n = pb.ns;
    return __ldg(pb.eri32 + ((p * n + q) * n + r) * n + s);
}
template <> __device__ __forceinline__ double load_eri<double>(const DevProblem& pb, int p, int q, int r, int s) {
    const int n = pb.ns;
    return __ldg(pb.eri64 + ((p * n + q) * n + r) * n + s);
}

// Correlator factor of moving two electrons (p1 -> x, p2 -> y; sf = 1 up, 2
// down for each move) given the two single-move factors r1, r2: correlators
// touched by both moves hold a site of each, so they are found through the
// site-pair lists and corrected to their joint new state.
template <typename R>
__device__ R corr_ratio_double(const DevProblem& pb, const uint32_t* cidx, int p1, int x, int p2, int y, R r1, R r2) {
    const int ns = pb.ns;
    const int sf1 = p1 >= ns ? 2 : 1, sf2 = p2 >= ns ? 2 : 1;
    const int a1[2] = {p1 % ns, x % ns}, a2[2] = {p2 % ns, y % ns};
    R corr = R(1);
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int i = a1[u], j = a2[v];
            // correlators holding a site of each move: the pair list of (i, j),
            // or every correlator on the site when both moves touch it
            const int lo = i == j ? pb.site_cptr[i] : pb.pair_ptr[i * ns + j];
            const int hi = i == j ? pb.site_cptr[i + 1] : pb.pair_ptr[i * ns + j + 1];
            for (int e = lo; e < hi; ++e) {
                const int c = i == j ? pb.site_corr[e] : pb.pair_corr[e];
                // counted once: skip if an earlier (u', v') combination also lies in c
                bool seen = false;
                for (int w = 0; w < u * 2 + v && !seen; ++w) {
                    const int i2 = a1[w >> 1], j2 = a2[w & 1];
                    seen = site_weight_in(pb, c, i2) != 0 && (i2 == j2 || site_weight_in(pb, c, j2) != 0);
                }
                if (seen) continue;
                const int old = (int)cidx[c];
                const int d1 = sf1 * (site_weight_in(pb, c, a1[1]) - site_weight_in(pb, c, a1[0]));
                const int d2 = sf2 * (site_weight_in(pb, c, a2[1]) - site_weight_in(pb, c, a2[0]));
                const int64_t o = pb.corr_off[c];
                const R c0 = load_C<R>(pb, o + old);
                corr *= load_C<R>(pb, o + old + d1 + d2) * c0 / (load_C<R>(pb, o + old + d1) * load_C<R>(pb, o + old + d2));
            }
        }
    return r1 * r2 * corr;
}

// Correlators of at most two sites (the pair correlators of the ab initio
// ansatz): the correlator factor of any move factorises over the sites it
// touches.  Rsite[4 s + v] = prod over the correlators c on site s of
// C_c(state with site s in local state v) / C_c(current state), all other
// sites unchanged.  A move that changes the local states of the distinct
// sites S (at most four) then has the factor prod_{s in S} Rsite[4 s + n'_s]
// times, for every correlator holding two sites s, t of S, the correction
// C(o + d_s + d_t) C(o) / (C(o + d_s) C(o + d_t)) (the two single-site
// factors each took the other site at its old state).
__device__ __forceinline__ int site_state(uint64_t up, uint64_t dn, int s) {
    return (int)((up >> s) & 1ull) + 2 * (int)((dn >> s) & 1ull);
}

template <typename R>
__device__ R pair_correction(const DevProblem& pb, const uint32_t* cidx, int s, int dvs, int t, int dvt) {
    R f = R(1);
    const int lo = pb.pair_ptr[s * pb.ns + t], hi = pb.pair_ptr[s * pb.ns + t + 1];
    for (int e = lo; e < hi; ++e) {
        const int c = pb.pair_corr[e];
        const int o = (int)cidx[c];
        const int ds = site_weight_in(pb, c, s) * dvs, dt = site_weight_in(pb, c, t) * dvt;
        const int64_t off = pb.corr_off[c];
        f *= load_C<R>(pb, off + o + ds + dt) * load_C<R>(pb, off + o) /
             (load_C<R>(pb, off + o + ds) * load_C<R>(pb, off + o + dt));
    }
    return f;
}

// The same correction from the sample's pair table: entry k(s, t) (s < t,
// row-major over site pairs) = the base C index corr_off[c] + state of the
// one correlator c holding s and t (bits 0-29, all ones if none) and whether
// s and t carry weight 4 in c (bits 30, 31).  Same arithmetic as the lists.
__device__ __forceinline__ int site_pair_index(int s, int t, int ns) { return s * (2 * ns - s - 1) / 2 + t - s - 1; }

template <typename R>
__device__ __forceinline__ R pair_correction_tab(const DevProblem& pb, const uint32_t* ptab, int s, int dvs, int t,
                                                 int dvt) {
    if (s > t) {
        const int u = s; s = t; t = u;
        const int d = dvs; dvs = dvt; dvt = d;
    }
    const uint32_t en = ptab[site_pair_index(s, t, pb.ns)];
    if (en == 0xFFFFFFFFu) return R(1);
    const int64_t off = (int64_t)(en & 0x3FFFFFFFu);
    const int ds = (((en >> 30) & 1u) ? 4 : 1) * dvs, dt = ((en >> 31) ? 4 : 1) * dvt;
    R f = R(1);
    f *= load_C<R>(pb, off + ds + dt) * load_C<R>(pb, off) / (load_C<R>(pb, off + ds) * load_C<R>(pb, off + dt));
    return f;
}

// factor of the move changing sites S[k] by D[k] (local state units), k < n
template <typename R>
__device__ __forceinline__ R site_move_factor(const DevProblem& pb, const uint32_t* cidx, const R* Rsite,
                                              const uint32_t* ptab, uint64_t up, uint64_t dn, int (&S)[4],
                                              int (&D)[4], int n) {
    bool alive[4] = {true, true, true, true};
    for (int k = 1; k < n; ++k)
        for (int m = 0; m < k; ++m)
            if (alive[m] && S[k] == S[m]) {
                D[m] += D[k];
                alive[k] = false;
                break;
            }
    R f = R(1);
    for (int k = 0; k < n; ++k)
        if (alive[k] && D[k] != 0) f *= Rsite[4 * S[k] + site_state(up, dn, S[k]) + D[k]];
    for (int k = 0; k < n; ++k)
        for (int m = k + 1; m < n; ++m)
            if (alive[k] && alive[m] && D[k] != 0 && D[m] != 0)
                f *= ptab ? pair_correction_tab<R>(pb, ptab, S[k], D[k], S[m], D[m])
                          : pair_correction<R>(pb, cidx, S[k], D[k], S[m], D[m]);
    return f;
}

// Local energy of the ab initio Hamiltonian for the warp's walker (lane
// partial sum; the caller reduces).  E_L = <n|H|n> + sum over single and
// double same-spin-conserving moves of <n|H|n'> Psi_n'/Psi_n.  With the new
// orbitals put in place of the old ones, the amplitude ratios are the
// in-place pfaffian ratios (their Jordan-Wigner signs cancel against those of
// the matrix elements, as for the hops) and the matrix elements are the
// Slater-Condon magnitudes:
//   single p->x:  h_px + sum_{k occ != p} [(px|kk) - d(s_k, s_p) (pk|kx)]
//   double p1->x, p2->y:  (p1 x|p2 y) - d(same spin) (p1 y|p2 x).
// Pfaffian ratios from G[q][j] = sum_k F[q][o_k] X[k][j] and, for doubles,
// H[y][x] = sum_j F[y][o_j] G[x][j] (second replacement on the rank-2-updated
// inverse, written out in G, X, F and H).
template <typename R>
__device__ double abinitio_energy(const DevProblem& pb, const R* X, int XS, const uint8_t* pos_orb,
                                  const int8_t* orb_pos, uint64_t up, uint64_t dn, const uint32_t* cidx,
                                  R* G, int GS, R* Hm, R* Rs, uint8_t* emp, int8_t* eidx, R* Rsite,
                                  uint32_t* ptab_s) {
    const bool pairs = pb.max_csites <= 2;   // the site-factorised correlator ratios apply
    const uint32_t* ptab = pairs && pb.pair_unique ? ptab_s : nullptr;
    const int lane = threadIdx.x & 31;
    const int ns = pb.ns, M = pb.M, N = pb.N, nu = pb.nu, nd = pb.nd;
    const int eu = ns - nu, ed = ns - nd, E = eu + ed;
    // empty orbitals: up first (ascending), then down
    for (int i = lane; i < E; i += 32)
        emp[i] = (uint8_t)(i < eu ? nth_set_bit64(~up & ((ns == 64) ? ~0ull : ((1ull << ns) - 1ull)), i)
                                  : ns + nth_set_bit64(~dn & ((ns == 64) ? ~0ull : ((1ull << ns) - 1ull)), i - eu));
    for (int o = lane; o < M; o += 32) eidx[o] = -1;
    __syncwarp();
    for (int i = lane; i < E; i += 32) eidx[emp[i]] = (int8_t)i;
    // G rows for every orbital
    for (int q = lane; q < M; q += 32) {
        for (int j = 0; j < N; ++j) G[q * GS + j] = R(0);
        for (int k = 0; k < N; ++k) {
            const R f = load_F<R>(pb, q, pos_orb[k]);
            for (int j = 0; j < N; ++j) G[q * GS + j] += f * X[k * XS + j];
        }
    }
    __syncwarp();
    // H over pairs of empty orbitals
    for (int t = lane; t < E * E; t += 32) {
        const int iy = t / E, ix = t % E;
        const int yq = emp[iy], xq = emp[ix];
        R acc = R(0);
        for (int j = 0; j < N; ++j) acc += load_F<R>(pb, yq, pos_orb[j]) * G[xq * GS + j];
        Hm[t] = acc;
    }
    if (pairs) {
        // per-site factors of every local state
        for (int t = lane; t < 4 * ns; t += 32) {
            const int s = t >> 2, v = t & 3, n = site_state(up, dn, s);
            R f = R(1);
            if (v != n)
                for (int ent = pb.site_cptr[s]; ent < pb.site_cptr[s + 1]; ++ent) {
                    const int c = pb.site_corr[ent];
                    const int64_t k = pb.corr_off[c] + (int64_t)cidx[c];
                    f *= load_C<R>(pb, k + pb.site_w[ent] * (v - n)) / load_C<R>(pb, k);
                }
            Rsite[t] = f;
        }
        if (ptab) {
            // the pair table of this sample (see pair_correction_tab)
            for (int si = 0; si + 1 < ns; ++si)
                for (int ti = si + 1 + lane; ti < ns; ti += 32) {
                    const int lo = pb.pair_ptr[si * ns + ti], hi = pb.pair_ptr[si * ns + ti + 1];
                    uint32_t en = 0xFFFFFFFFu;
                    if (hi > lo) {
                        const int c = pb.pair_corr[lo];
                        en = (uint32_t)(pb.corr_off[c] + (int64_t)cidx[c]) |
                             (site_weight_in(pb, c, si) == 4 ? 1u << 30 : 0u) |
                             (site_weight_in(pb, c, ti) == 4 ? 1u << 31 : 0u);
                    }
                    ptab_s[site_pair_index(si, ti, ns)] = en;
                }
        }
    } else {
        // single-move correlator factors Rs[a][ie] (same spin only)
        for (int t = lane; t < N * E; t += 32) {
            const int a = t / E, ie = t % E;
            const int p = pos_orb[a], q = emp[ie];
            Rs[t] = ((p >= ns) == (q >= ns)) ? corr_ratio_serial<R>(pb, cidx, p, q) : R(0);
        }
    }
    __syncwarp();
    double e = 0.0;
    // diagonal: sum_k h_kk + 1/2 sum_{k != l} [(kk|ll) - d(s_k, s_l) (kl|lk)]
    for (int a = lane; a < N; a += 32) {
        const int k = pos_orb[a], ik = k % ns;
        double v = (double)load_h<R>(pb, ik, ik);
        for (int b = 0; b < N; ++b) {
            if (b == a) continue;
            const int l = pos_orb[b], il = l % ns;
            R w = load_eri<R>(pb, ik, ik, il, il);
            if ((k >= ns) == (l >= ns)) w -= load_eri<R>(pb, ik, il, il, ik);
            v += 0.5 * (double)w;
        }
        e += v;
    }
    // singles
    for (int t = lane; t < N * E; t += 32) {
        const int a = t / E, ie = t % E;
        const int p = pos_orb[a], x = emp[ie];
        if ((p >= ns) != (x >= ns)) continue;
        const int ip = p % ns, ix = x % ns;
        R hm = load_h<R>(pb, ip, ix);
        for (int b = 0; b < N; ++b) {
            if (b == a) continue;
            const int k = pos_orb[b], ik = k % ns;
            hm += load_eri<R>(pb, ip, ix, ik, ik);
            if ((k >= ns) == (p >= ns)) hm -= load_eri<R>(pb, ip, ik, ik, ix);
        }
        R rc;
        if (pairs) {
            const int sf = p >= ns ? 2 : 1;
            int S[4] = {ip, ix, 0, 0}, D[4] = {-sf, sf, 0, 0};
            rc = site_move_factor<R>(pb, cidx, Rsite, ptab, up, dn, S, D, 2);
        } else {
            rc = Rs[t];
        }
        e += (double)(hm * G[x * GS + a] * rc);
    }
    // doubles: up-up, down-down and up-down classes.  Within a class the
    // lanes run over (electron pair, empty pair) with the electron pair
    // outer; both pairs come from the host's tables (dexc), the position in
    // each advancing by 32 per step.
    {
        const int nab[3] = {nu * (nu - 1) / 2, nd * (nd - 1) / 2, nu * nd};
        const int nxy[3] = {eu * (eu - 1) / 2, ed * (ed - 1) / 2, eu * ed};
        term_sum<R> ed;
        const uint16_t* tab_ab = pb.dexc;
        const uint16_t* tab_xy = pb.dexc + nab[0] + nab[1] + nab[2];
        for (int cls = 0; cls < 3; ++cls) {
            const int nx = nxy[cls], total = nab[cls] * nx;
            if (cls > 0) {
                tab_ab += nab[cls - 1];
                tab_xy += nxy[cls - 1];
            }
            if (total == 0) continue;
            int kab = lane / nx, kxy = lane - (lane / nx) * nx;
            for (int t = lane; t < total; t += 32) {
                const uint32_t ab = tab_ab[kab], xy = tab_xy[kxy];
                kxy += 32;
                while (kxy >= nx) {
                    kxy -= nx;
                    ++kab;
                }
                const int a = (int)(ab & 255u), b = (int)(ab >> 8), ix = (int)(xy & 255u), iy = (int)(xy >> 8);
                const int p1 = pos_orb[a], p2 = pos_orb[b], x = emp[ix], y = emp[iy];
                const int i1 = p1 >= ns ? p1 - ns : p1, i2 = p2 >= ns ? p2 - ns : p2;
                const int jx = x >= ns ? x - ns : x, jy = y >= ns ? y - ns : y;
                R hm = load_eri<R>(pb, i1, jx, i2, jy);
                if ((p1 >= ns) == (p2 >= ns)) hm -= load_eri<R>(pb, i1, jy, i2, jx);
                if (hm == R(0)) continue;
                // pfaffian ratio for a -> x then b -> y
                const R Xab = X[a * XS + b], Xba = X[b * XS + a];
                const R Gxa = G[x * GS + a], Gxb = G[x * GS + b], Gya = G[y * GS + a], Gyb = G[y * GS + b];
                const R Fyp1 = load_F<R>(pb, y, p1), Fyp2 = load_F<R>(pb, y, p2), Fyx = load_F<R>(pb, y, x);
                const R Fxp1 = load_F<R>(pb, x, p1);
                const R r1 = Gxa;
                const R T1 = Gyb - Fyp1 * Xab + Fyx * Xab;
                const R Sc = Gya - Fyp2 * Xba;
                const R ytb = -Gxb + Fxp1 * Xab;
                const R Sy = -(Hm[iy * E + ix] - Fyp1 * Gxa - Fyp2 * Gxb) + Fxp1 * (-Gya - Fyp2 * Xab) +
                             Fyx * (R(1) - r1);
                const R rpf = r1 * T1 + Sc * ytb - Sy * Xba;
                R rc;
                if (pairs) {
                    const int sf1 = p1 >= ns ? 2 : 1, sf2 = p2 >= ns ? 2 : 1;
                    int S[4] = {i1, jx, i2, jy}, D[4] = {-sf1, sf1, -sf2, sf2};
                    rc = site_move_factor<R>(pb, cidx, Rsite, ptab, up, dn, S, D, 4);
                } else {
                    rc = corr_ratio_double<R>(pb, cidx, p1, x, p2, y, Rs[a * E + ix], Rs[b * E + iy]);
                }
                ed.add(hm * rpf * rc);
            }
        }
        e += ed.value();
    }
    return e;
}

// X = F[o, o]^{-1} for the current (unsorted) positions o, from scratch
template <typename R>
__device__ bool rebuild_inverse(const DevProblem& pb, R* X, int N, int XS, const uint8_t* pos_orb, R* col,
                                uint8_t* piv) {
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < N; ++i) {
        int p = pos_orb[i];
        for (int j = lane; j < N; j += 32) X[i * XS + j] = load_F<R>(pb, p, pos_orb[j]);
    }
    __syncwarp();
    return gj_invert_warp<R>(X, N, XS, col, piv);
}

template <typename R> __device__ __forceinline__ void store_pf(const SampleArgs& a, int64_t idx, R w);
template <> __device__ __forceinline__ void store_pf<float>(const SampleArgs& a, int64_t idx, float w) {
    if (a.s_pf64) a.s_pf64[idx] = (double)w;
    if (a.s_pf32) a.s_pf32[idx] = w;
    if (a.s_pf16) a.s_pf16[idx] = __float2bfloat16_rn(w);
}
template <> __device__ __forceinline__ void store_pf<double>(const SampleArgs& a, int64_t idx, double w) {
    if (a.s_pf64) a.s_pf64[idx] = w;
    if (a.s_pf32) a.s_pf32[idx] = (float)w;
    if (a.s_pf16) a.s_pf16[idx] = __float2bfloat16_rn((float)w);
}

// One walker (or one given configuration) of the problem of `a`, run by the
// calling warp with its shared-memory slice `base`.
template <typename R>
__device__ void walker_run(const SampleArgs& a, int w, unsigned char* base) {
    const DevProblem& pb = a.pb;
    const int lane = threadIdx.x & 31;
    const int N = pb.N, M = pb.M, ns = pb.ns, nu = pb.nu, XS = a.XS;
    R* X = (R*)base;
    R* bv = X + N * XS;
    R* yv = bv + XS;
    R* cv = yv + XS;
    uint8_t* iv = (uint8_t*)(cv + XS);         // 64 positions
    uint32_t* cidx = (uint32_t*)(iv + 64);     // ncorr (rounded up to 4)
    uint8_t* pos_orb = (uint8_t*)(cidx + a.ncorr_pad);
    int8_t* orb_pos = (int8_t*)(pos_orb + 64); // 128

    // ---- load the configuration -----------------------------------------
    for (int o = lane; o < M; o += 32) orb_pos[o] = -1;
    __syncwarp();
    uint64_t up = 0, dn = 0;
    bool bad = false;
    for (int i = lane; i < N; i += 32) {
        int o = a.walker_occ[(int64_t)w * N + i];
        pos_orb[i] = (uint8_t)o;
        if (o >= M) bad = true;
        else if (o < ns) up |= 1ull << o;
        else dn |= 1ull << (o - ns);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        up |= __shfl_xor_sync(VMC_FULL_MASK, up, o);
        dn |= __shfl_xor_sync(VMC_FULL_MASK, dn, o);
    }
    bad = __any_sync(VMC_FULL_MASK, bad);
    if (bad || __popcll(up) != nu || __popcll(dn) != pb.nd) {
        if (lane == 0) atomicOr(a.status, ST_BAD_CONFIG);
        return;
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) orb_pos[pos_orb[i]] = (int8_t)i;
    __syncwarp();

    // ---- inverse of the pairing submatrix, from scratch -------------------
    if (!rebuild_inverse<R>(pb, X, N, XS, pos_orb, cv, iv)) {
        if (lane == 0) atomicOr(a.status, ST_SINGULAR);
        return;
    }

    // ---- correlator states --------------------------------------------------
    for (int c = lane; c < pb.ncorr; c += 32) {
        uint32_t idx = 0, wgt = 1;
        for (int j = pb.corr_ptr[c]; j < pb.corr_ptr[c + 1]; ++j) {
            int s = pb.corr_sites[j];
            idx += wgt * (uint32_t)(((up >> s) & 1ull) + 2ull * ((dn >> s) & 1ull));
            wgt <<= 2;
        }
        cidx[c] = idx;
    }
    __syncwarp();

    const uint64_t sitemask = (ns == 64) ? ~0ull : ((1ull << ns) - 1ull);
    uint64_t step = a.walker_step ? a.walker_step[w] : 0ull;
    double lnrun = 0.0;   // ln|Psi| of the chain relative to its start, summed from the accepted ratios
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int n_sweeps = a.n_burn + a.spw;
    // Philox words of 32 consecutive proposals at once: lane L holds those of
    // counter step0 + L, and each proposal reads its own by shuffle (the same
    // numbers as one evaluation per proposal, a 32nd of the instructions)
    uint64_t step0 = step;
    u32x4 rl = philox4x32_10(u32x4{(uint32_t)w, (uint32_t)(step0 + lane), (uint32_t)((step0 + lane) >> 32), 0u},
                             k0, k1);

    for (int sw = 0; sw < n_sweeps; ++sw) {
        for (int t = 0; t < a.props_per_sweep; ++t) {
            if (step - step0 >= 32u) {
                step0 = step;
                const uint64_t sl = step0 + (uint64_t)lane;
                rl = philox4x32_10(u32x4{(uint32_t)w, (uint32_t)sl, (uint32_t)(sl >> 32), 0u}, k0, k1);
            }
            const int rsrc = (int)(step - step0);
            u32x4 r;
            r.x = __shfl_sync(VMC_FULL_MASK, rl.x, rsrc);
            r.y = __shfl_sync(VMC_FULL_MASK, rl.y, rsrc);
            r.z = __shfl_sync(VMC_FULL_MASK, rl.z, rsrc);
            ++step;
            int as = (int)mulhi32(r.x, (uint32_t)N);
            int p = as < nu ? nth_set_bit64(up, as) : ns + nth_set_bit64(dn, as - nu);
            int spin = p >= ns;
            uint64_t m = spin ? dn : up;
            int n_empty = ns - __popcll(m);
            if (n_empty <= 0) continue;
            int kk = (int)mulhi32(r.y, (uint32_t)n_empty);
            int q = spin * ns + nth_set_bit64(~m & sitemask, kk);
            R u = R(r.z >> 8) * R(1.0 / 16777216.0);
            int ap = orb_pos[p];
            // correlator factor, one membership entry per lane when the two
            // sites have at most 32: its two parameter loads (L2) go out
            // first and are waited on after the pfaffian row product
            const int csf = spin + 1, csp = p - spin * ns, csq = q - spin * ns;
            const int ctot = (pb.site_cptr[csp + 1] - pb.site_cptr[csp]) + (pb.site_cptr[csq + 1] - pb.site_cptr[csq]);
            const bool cfast = ctot <= 32;
            R cnum = R(1), cden = R(1);
            int cc = -1, cnew = -1;
            if (cfast && lane < ctot) {
                cnew = corr_entry(pb, cidx, csp, csq, csf, lane, &cc);
                if (cc >= 0) {
                    cnum = load_C<R>(pb, pb.corr_off[cc] + cnew);
                    cden = load_C<R>(pb, pb.corr_off[cc] + cidx[cc]);
                }
            }
            R acc = R(0);
            for (int j = lane; j < N; j += 32) {
                R bj = (j == ap) ? R(0) : load_F<R>(pb, q, pos_orb[j]);
                bv[j] = bj;
                acc += bj * X[ap * XS + j];
            }
            R rpf = -warp_sum(acc);
            R rc = cfast ? warp_prod(cnum / cden) : corr_ratio_warp<R>(pb, cidx, p, q, false);
            R ratio = rpf * rc;
            bool accept = u < ratio * ratio;
            if (!accept) continue;
            lnrun += (double)log_abs(ratio);
            __syncwarp();
            {
                // lane L owns the column pair 2L, 2L + 1 (XS even); X is
                // antisymmetric, so c = X[:, a] = -X[a, :] and
                // y_j = (X b)_j + [j = a] = -sum_i b_i X_ij + [j = a]
                using R2 = typename pair_of<R>::type;
                const int j0 = 2 * lane;
                const bool own = j0 < N;
                R2* cy = reinterpret_cast<R2*>(yv);   // (c_i / r, y_i / r) of every row
                R2 cj{R(0), R(0)}, yj{R(0), R(0)};
                const R rinv = R(1) / rpf;
                if (own) {
                    const R2 xa = *reinterpret_cast<const R2*>(X + ap * XS + j0);
                    cj.x = -xa.x;
                    cj.y = -xa.y;
                    for (int i = 0; i < N; ++i) {
                        const R bi = bv[i];
                        const R2 x = *reinterpret_cast<const R2*>(X + i * XS + j0);
                        yj.x = fma(-bi, x.x, yj.x);
                        yj.y = fma(-bi, x.y, yj.y);
                    }
                    if (j0 == ap) yj.x += R(1);
                    if (j0 + 1 == ap) yj.y += R(1);
                    cy[j0] = R2{cj.x * rinv, yj.x * rinv};
                    if (j0 + 1 < N) cy[j0 + 1] = R2{cj.y * rinv, yj.y * rinv};
                }
                __syncwarp();
                if (own) {
                    // X_ij += (c_i y_j - y_i c_j) / r
                    for (int i = 0; i < N; ++i) {
                        const R2 ci = cy[i];
                        R2* xp = reinterpret_cast<R2*>(X + i * XS + j0);
                        R2 x = *xp;
                        x.x = fma(ci.x, yj.x, fma(-ci.y, cj.x, x.x));
                        x.y = fma(ci.x, yj.y, fma(-ci.y, cj.y, x.y));
                        *xp = x;
                    }
                }
            }
            if (cfast) {
                __syncwarp();
                if (cc >= 0) cidx[cc] = (uint32_t)cnew;
                __syncwarp();
            } else {
                corr_ratio_warp<R>(pb, cidx, p, q, true);
            }
            if (lane == 0) {
                pos_orb[ap] = (uint8_t)q;
                orb_pos[p] = -1;
                orb_pos[q] = (int8_t)ap;
            }
            if (spin) dn = (dn & ~(1ull << (p - ns))) | (1ull << (q - ns));
            else up = (up & ~(1ull << p)) | (1ull << q);
            __syncwarp();
        }
        // periodic from-scratch rebuild bounds the drift of the rank-2 updates
        if (a.refresh_every > 0 && a.props_per_sweep > 0 && (sw + 1) % a.refresh_every == 0) {
            if (!rebuild_inverse<R>(pb, X, N, XS, pos_orb, cv, iv)) {
                if (lane == 0) atomicOr(a.status, ST_SINGULAR);
                return;
            }
        }
        if (sw < a.n_burn) continue;

        // ---- measurement ----------------------------------------------------
        const int64_t s = (int64_t)w * a.spw + (sw - a.n_burn);
        double e_lane = 0.0;
        if (a.want_energy) {
            if (pb.ham == 0) {
                for (int i = lane; i < N; i += 32) {
                    int p = pos_orb[i];
                    int spin = p >= ns;
                    int sp = p - spin * ns;
                    uint64_t m = spin ? dn : up;
                    for (int k = pb.nbr_ptr[sp]; k < pb.nbr_ptr[sp + 1]; ++k) {
                        int s2 = pb.nbr_site[k];
                        if ((m >> s2) & 1ull) continue;
                        int q = spin * ns + s2;
                        R d = R(0);
#pragma unroll 8
                        for (int j = 0; j < N; ++j)
                            if (j != i) d += load_F<R>(pb, q, pos_orb[j]) * X[i * XS + j];
                        R rc = corr_ratio_serial<R>(pb, cidx, p, q);
                        // -t * (Pf ratio = -d) * rc
                        e_lane += pb.nbr_t[k] * (double)(d * rc);
                    }
                }
            }
            if (pb.ham == 1) {
                unsigned char* ab = (unsigned char*)(orb_pos + 128);
                R* G = (R*)ab;
                R* Hm = G + (size_t)M * a.GS;
                R* Rs = Hm + (size_t)(M - N) * (M - N);
                uint8_t* emp = (uint8_t*)(Rs + (size_t)N * (M - N));
                int8_t* eidx = (int8_t*)(emp + 128);
                R* Rsite = (R*)(eidx + 128);
                uint32_t* ptab = (uint32_t*)(Rsite + 4 * ns);
                e_lane = abinitio_energy<R>(pb, X, XS, pos_orb, orb_pos, up, dn, cidx, G, a.GS, Hm, Rs, emp, eidx,
                                            Rsite, ptab);
                __syncwarp();
            }
            e_lane = warp_sum(e_lane);
            if (pb.ham == 0) e_lane += pb.U * (double)__popcll(up & dn);
            if (!isfinite(e_lane) && lane == 0) atomicOr(a.status, ST_NONFINITE);
        }
        // ascending occupation and the position of each sorted electron
        for (int i = lane; i < N; i += 32) {
            int o = i < nu ? nth_set_bit64(up, i) : ns + nth_set_bit64(dn, i - nu);
            iv[i] = (uint8_t)orb_pos[o];
            if (a.s_occ) a.s_occ[s * a.Nst + i] = (uint8_t)o;
        }
        __syncwarp();
        if (a.bgrad) {
            // adjoint: grad += w_s O(n_s)
            double ws = a.bw[s];
            for (int c = lane; c < pb.ncorr; c += 32) {
                int64_t k = pb.corr_off[c] + cidx[c];
                atomicAdd(a.bgrad + k, ws / pb.C64[k]);
            }
            for (int e = lane; e < pb.P; e += 32) {
                uint16_t t = pb.pairtab[e];
                int aa = t & 255, bb = t >> 8;
                int oa = pos_orb[iv[aa]], ob = pos_orb[iv[bb]];
                atomicAdd(a.bgrad + pb.ncp + pb.rowbase[oa] + ob, ws * (double)X[iv[bb] * XS + iv[aa]]);
            }
        } else {
            if (a.s_E && lane == 0) a.s_E[s] = e_lane;
            if (a.s_lnrun && lane == 0) a.s_lnrun[s] = lnrun;
            if (a.s_cidx)
                for (int c = lane; c < pb.ncorr; c += 32) a.s_cidx[s * a.ncst + c] = (cstate_t)cidx[c];
            for (int e = lane; e < pb.P; e += 32) {
                uint16_t t = pb.pairtab[e];
                int aa = t & 255, bb = t >> 8;
                store_pf<R>(a, s * a.Pst + e, X[iv[bb] * XS + iv[aa]]);
            }
        }
        __syncwarp();
    }

    // ---- write the chain state back (ascending) ------------------------------
    if (a.write_back) {
        for (int i = lane; i < N; i += 32) {
            int o = i < nu ? nth_set_bit64(up, i) : ns + nth_set_bit64(dn, i - nu);
            a.walker_occ[(int64_t)w * N + i] = (uint8_t)o;
        }
        if (lane == 0 && a.walker_step) a.walker_step[w] = step;
    }
}

template <typename R>
__global__ void k_walkers(SampleArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = threadIdx.x >> 5;
    const int w = blockIdx.x * (blockDim.x >> 5) + wid;
    if (w >= a.n_walkers) return;
    walker_run<R>(a, w, smem_raw + (size_t)wid * a.warp_bytes);
}

// Several problems (lattices of uneven size) in one launch: warp g runs
// walker g - wstart[b] of problem b, wstart[b] <= g < wstart[b + 1]; every
// warp has warp_bytes of shared memory (the largest of the problems').
template <typename R>
__global__ void k_walkers_batch(const SampleArgs* __restrict__ args, const int* __restrict__ wstart, int n,
                                size_t warp_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = threadIdx.x >> 5;
    const int g = blockIdx.x * (blockDim.x >> 5) + wid;
    if (g >= wstart[n]) return;
    int b = 0;
    while (b + 1 < n && g >= wstart[b + 1]) ++b;
    walker_run<R>(args[b], g - wstart[b], smem_raw + (size_t)wid * warp_bytes);
}

// ln|Pf(F[occ, occ])| + sum_c ln|C_c| per sample, FP64 Parlett-Reid with
// pivoting (the pfaffian reduction cited in Sec. II.C), one warp per sample.
__global__ void k_logpsi(LogPsiArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevProblem& pb = a.pb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (s >= a.n_s) return;
    const int N = pb.N, XS = a.XS;
    double* A = (double*)(smem_raw + (size_t)wid * a.warp_bytes);
    double* tau = A + N * XS;
    double* colk1 = tau + XS;
    const uint8_t* occ = a.s_occ + s * a.Nst;
    for (int i = 0; i < N; ++i)
        for (int j = lane; j < N; j += 32) A[i * XS + j] = __ldg(pb.F64 + occ[i] * pb.M + occ[j]);
    __syncwarp();
    double logabs = 0.0;
    int sign = 1;
    for (int k = 0; k + 1 < N; k += 2) {
        double best = -1.0;
        int bi = N;
        for (int i = k + 1 + lane; i < N; i += 32) {
            double v = fabs(A[i * XS + k]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(VMC_FULL_MASK, best, o);
            int oi = __shfl_xor_sync(VMC_FULL_MASK, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0)) { sign = 0; break; }
        if (bi != k + 1) {
            for (int j = lane; j < N; j += 32) {
                double t = A[(k + 1) * XS + j];
                A[(k + 1) * XS + j] = A[bi * XS + j];
                A[bi * XS + j] = t;
            }
            __syncwarp();
            for (int i = lane; i < N; i += 32) {
                double t = A[i * XS + k + 1];
                A[i * XS + k + 1] = A[i * XS + bi];
                A[i * XS + bi] = t;
            }
            sign = -sign;
        }
        __syncwarp();
        double piv = A[k * XS + k + 1];
        if (piv < 0) sign = -sign;
        logabs += log(fabs(piv));
        for (int i = k + 2 + lane; i < N; i += 32) {
            tau[i] = A[k * XS + i] / piv;
            colk1[i] = A[i * XS + k + 1];
        }
        __syncwarp();
        for (int j = k + 2 + lane; j < N; j += 32) {
            double tj = tau[j], cj = colk1[j];
            for (int i = k + 2; i < N; ++i) A[i * XS + j] += tau[i] * cj - colk1[i] * tj;
        }
        __syncwarp();
    }
    // correlators
    const cstate_t* ci = a.s_cidx + s * a.ncst;
    double lc = 0.0;
    for (int c = lane; c < pb.ncorr; c += 32) {
        double v = pb.C64[pb.corr_off[c] + ci[c]];
        lc += log(fabs(v));
    }
    lc = warp_sum(lc);
    if (lane == 0) a.out[s] = sign == 0 ? -INFINITY : logabs + lc;
}

template __global__ void k_walkers<float>(SampleArgs);
template __global__ void k_walkers<double>(SampleArgs);

// launch of the batched walker kernel from the unit that defines it
cudaError_t launch_walkers_batch(bool fp64, int blocks, int threads, size_t smem, cudaStream_t st,
                                 const SampleArgs* args, const int* wstart, int n, size_t warp_bytes) {
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(k_walkers_batch<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_walkers_batch<double><<<blocks, threads, smem, st>>>(args, wstart, n, warp_bytes);
    } else {
        e = cudaFuncSetAttribute(k_walkers_batch<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_walkers_batch<float><<<blocks, threads, smem, st>>>(args, wstart, n, warp_bytes);
    }
    return cudaGetLastError();
}

}  // namespace vmc
