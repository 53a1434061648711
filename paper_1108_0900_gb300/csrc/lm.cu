// Accelerated linear method (Sec. II.B): the products of the matrices of
// Eq. 8 with a vector x = (x_0, x_1 .. x_nv) over the basis
// {Psi, Psi^1 .. Psi^nv}, evaluated from the stored samples by Eq. 10 with
// the Hamiltonian in the factored form of Eq. 9,
//   H = c0 + sum_mu Lhat_mu Rhat_mu,  Lhat_mu = sum_ij L^mu_ij E_ij,
//   E_ij = sum_sigma a+_{i sigma} a_{j sigma}:
//   (H x)_i = (1/n) sum_n sum_pq Q_{n q p i} z_pq(n) + c0 (S x)_i,
//   z_pq = sum_mu L^mu_pq w_mu,  w_mu = sum_rs R^mu_rs y_rs,
//   y_rs = sum_j Q_{n r s j} x_j,  Q_{n r s j} = <n| a+_r a_s |Psi^j> / Psi_n,
//   (S x)_i = (1/n) sum_n O_i(n) (x_0 + O(n) . x).
//
// One warp owns one sample.  Q_{n r s j} is nonzero for r occupied in n and
// s = r (then Q = O_j(n), O_0 = 1) or s empty with the spin of r (then n'
// = n with the electron at r moved to s and Q = rho Psi^j_n' / Psi_n').  The
// signed amplitude ratio of the move of the electron at sorted position a
// to the empty orbital v is rho = rho_c G[v][a], G = F[:, occ] A^{-1},
// A = F[occ, occ] (the in-place pfaffian ratio, whose sign includes the
// Jordan-Wigner sign of the hop), rho_c the correlator ratio.  Contracting
// with x never forms O(n'): sum_j Q_{n r s j} x_j is the derivative of
// rho Psi_n along x, divided by Psi_n,
//   y = rho_c (G[v][a] (x_0 + O(n).x + dln rho_c) + D[v][a]),
//   D = (X[:, occ] - G X[occ, occ]) A^{-1}    (dG along x; X = the pairing
//                                               part of x as an antisymmetric
//                                               matrix),
// and the transposed contraction sum_pq Q_{n q p i} z_pq is its adjoint:
// with c_e = z_e rho_c per move e and B = Cbar A^{-T} (Cbar[v][a] = c_e),
// the pairing amplitude f_uw collects B[v][k] at (v, o_k) and -(G^T B)[l][k]
// at (o_l, o_k), antisymmetrised, plus W O(n) with W = sum of z rho over all
// moves (and the diagonal terms), and the correlators collect
// c_e G (1/C at the new state - 1/C at the old one).  Per sample: five
// (M - N) x N x N products in shared memory, two contractions with the
// factors (kept as sparse matrices: the Hubbard ones are diagonal or follow
// the bonds) and one atomic add per touched parameter.
#include "ansatz.cuh"
#include "common.cuh"
#include "kernels.h"

namespace vmc {

namespace {

// Correlator part of the ratio for moving the electron at spin orbital p to
// q, and the derivative of its logarithm along x (xc = x_k / C_k):
// sum over the correlators that change of xc[new state] - xc[old state].
template <typename R>
__device__ R corr_ratio_dir(const DevProblem& pb, const uint32_t* cidx, int p, int q, const R* xc, R* dl) {
    const int ns = pb.ns;
    const int sf = p >= ns ? 2 : 1;
    const int sp = p >= ns ? p - ns : p, sq = q >= ns ? q - ns : q;
    const int total = (pb.site_cptr[sp + 1] - pb.site_cptr[sp]) + (pb.site_cptr[sq + 1] - pb.site_cptr[sq]);
    R prod = R(1), d = R(0);
    for (int e = 0; e < total; ++e) {
        int c;
        const int newi = corr_entry(pb, cidx, sp, sq, sf, e, &c);
        if (c < 0) continue;
        const int64_t k1 = pb.corr_off[c] + newi, k0 = pb.corr_off[c] + cidx[c];
        prod *= load_C<R>(pb, k1) / load_C<R>(pb, k0);
        d += xc[k1] - xc[k0];
    }
    *dl = d;
    return prod;
}

// Adjoint of the correlator ratio: coef (1/C at the new state) and
// -coef (1/C at the old state) for every correlator the move changes.  The
// old-state parts of all moves of a sample share one parameter per
// correlator, so they are summed per correlator in shared memory (old[c])
// and leave with the sample's own O(n) term: one global atomic per
// correlator instead of one per move.
template <typename R>
__device__ void corr_ratio_adjoint(const DevProblem& pb, const uint32_t* cidx, int p, int q, double coef,
                                   double* out, R* old) {
    const int ns = pb.ns;
    const int sf = p >= ns ? 2 : 1;
    const int sp = p >= ns ? p - ns : p, sq = q >= ns ? q - ns : q;
    const int total = (pb.site_cptr[sp + 1] - pb.site_cptr[sp]) + (pb.site_cptr[sq + 1] - pb.site_cptr[sq]);
    for (int e = 0; e < total; ++e) {
        int c;
        const int newi = corr_entry(pb, cidx, sp, sq, sf, e, &c);
        if (c < 0) continue;
        const int64_t k1 = pb.corr_off[c] + newi;
        atomicAdd(out + k1, coef / __ldg(pb.C64 + k1));
        atomicAdd(old + c, (R)coef);
    }
}

// move t of the same-spin list: up electrons to up holes, then down to down
__device__ __forceinline__ void decode_move(int t, int nu, int eu, int ed, int* a, int* ie) {
    const int nup = nu * eu;
    if (t < nup) {
        *a = t / eu;
        *ie = t % eu;
    } else {
        const int u = t - nup;
        *a = nu + u / ed;
        *ie = eu + u % ed;
    }
}

// C (+)= alpha A B over one warp with T x T register tiles per lane:
// A(i, k) = A[i sai + k sak], B(k, j) = B[k sbk + j sbj], C[i sc + j]; i < m,
// j < n, k < K.  Ragged tiles clamp their loads and skip their stores.
template <typename R, int T>
__device__ void warp_gemm(int m, int n, int K, const R* A, int sai, int sak, const R* B, int sbk, int sbj, R* C,
                          int sc, R alpha, bool accumulate) {
    const int lane = threadIdx.x & 31;
    const int tn = (n + T - 1) / T, nt = ((m + T - 1) / T) * tn;
    for (int tile = lane; tile < nt; tile += 32) {
        const int i0 = (tile / tn) * T, j0 = (tile % tn) * T;
        const R* Ar[T];
        const R* Bc[T];
#pragma unroll
        for (int r = 0; r < T; ++r) Ar[r] = A + min(i0 + r, m - 1) * sai;
#pragma unroll
        for (int c = 0; c < T; ++c) Bc[c] = B + min(j0 + c, n - 1) * sbj;
        R acc[T][T];
#pragma unroll
        for (int r = 0; r < T; ++r)
#pragma unroll
            for (int c = 0; c < T; ++c) acc[r][c] = R(0);
        for (int k = 0; k < K; ++k) {
            R av[T], bv[T];
#pragma unroll
            for (int r = 0; r < T; ++r) av[r] = Ar[r][k * sak];
#pragma unroll
            for (int c = 0; c < T; ++c) bv[c] = Bc[c][k * sbk];
#pragma unroll
            for (int r = 0; r < T; ++r)
#pragma unroll
                for (int c = 0; c < T; ++c) acc[r][c] += av[r] * bv[c];
        }
#pragma unroll
        for (int r = 0; r < T; ++r)
#pragma unroll
            for (int c = 0; c < T; ++c)
                if (i0 + r < m && j0 + c < n) {
                    R* q = C + (i0 + r) * sc + j0 + c;
                    *q = accumulate ? *q + alpha * acc[r][c] : alpha * acc[r][c];
                }
    }
}

}  // namespace

size_t lm_warp_bytes(int N, int M, int ns, int n_mu, int ncorr, int elem) {
    const size_t XS = N + 1, GS = N + 1, E = M - N;
    const size_t nmove = (size_t)(N / 2 + 1) * (size_t)(M - N + 2);   // >= nu eu + nd ed
    const size_t nr = 2 * N * XS + 3 * E * GS + (size_t)ns * ns + (size_t)((n_mu + 1) / 2 * 2) +
                      (size_t)((ncorr + 1) / 2 * 2) + (nmove + 1) / 2 * 2;
    const size_t b = nr * elem + (size_t)((ncorr + 3) / 4 * 4) * 4 + 64 + 128;
    return (b + 15) / 16 * 16;
}

// x -> the antisymmetric matrix of its pairing part and x_k / C_k
template <typename R>
__global__ void k_lm_prep(DevProblem pb, const double* x, R* Xt, R* xc) {
    const int64_t MM = (int64_t)pb.M * pb.M;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < MM + pb.ncp;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < MM) {
            const int p = (int)(t / pb.M), q = (int)(t % pb.M);
            double v = 0.0;
            if (p < q) v = x[1 + pb.ncp + pb.rowbase[p] + q];
            else if (p > q) v = -x[1 + pb.ncp + pb.rowbase[q] + p];
            Xt[t] = (R)v;
        } else {
            const int64_t k = t - MM;
            xc[k] = (R)(x[1 + k] / pb.C64[k]);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_lm_apply(LmArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DevProblem& pb = a.pb;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int N = pb.N, M = pb.M, ns = pb.ns, nu = pb.nu, nd = pb.nd, ncorr = pb.ncorr;
    const int eu = ns - nu, ed = ns - nd, E = eu + ed;
    const int XS = a.XS, GS = a.GS, n_mu = a.n_mu, nn = ns * ns;
    R* X = (R*)(smem_raw + (size_t)wid * a.warp_bytes);   // A^{-1}, sorted positions
    R* G = X + N * XS;                                      // G[ie][a], rows = empty orbitals
    R* Xo = G + E * GS;                                     // X[o_l][o_k], later G^T B
    R* Pm = Xo + N * XS;                                    // X[v][o_k] - (G Xo)[v][k], later Cbar
    R* D = Pm + E * GS;                                     // P A^{-1}, later B = Cbar A^{-T}
    R* Y = D + E * GS;                                      // y summed over spins, later z
    R* w = Y + nn;
    R* cold = w + (n_mu + 1) / 2 * 2;                       // old-state adjoint sums per correlator
    R* rcm = cold + (ncorr + 1) / 2 * 2;                    // correlator ratio of every move
    const int nmove = (N / 2 + 1) * (M - N + 2);
    uint32_t* cidx = (uint32_t*)(rcm + (nmove + 1) / 2 * 2);
    uint8_t* occ = (uint8_t*)(cidx + (ncorr + 3) / 4 * 4);
    uint8_t* emp = occ + 64;
    const R* Xt = (const R*)a.Xt;
    const R* xc = (const R*)a.xc;
    const R* Lval = (const R*)a.Lval;
    const R* Rval = (const R*)a.Rval;
    const R* pf = (const R*)a.pf;
    const R x0 = (R)a.x[0];
    const R c0 = (R)a.c0;
    const double sc = a.inv_n;
    const int nex = nu * eu + nd * ed;
    const uint64_t smask = ns == 64 ? ~0ull : ((1ull << ns) - 1ull);
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    double* Hf = a.Hx + 1 + pb.ncp;

    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; s < a.n_s; s += nwarps) {
        // ---- configuration, A^{-1} and O(n) . x ---------------------------
        uint64_t up = 0, dn = 0;
        for (int i = 0; i < N; ++i) {
            const int o = a.s_occ[s * a.Nst + i];
            if (lane == 0) occ[i] = (uint8_t)o;
            if (o < ns) up |= 1ull << o;
            else dn |= 1ull << (o - ns);
        }
        for (int c = lane; c < ncorr; c += 32) cidx[c] = (uint32_t)a.s_cidx[s * a.ncst + c];
        for (int i = lane; i < E; i += 32)
            emp[i] = (uint8_t)(i < eu ? nth_set_bit64(~up & smask, i) : ns + nth_set_bit64(~dn & smask, i - eu));
        for (int e = lane; e < pb.P; e += 32) {
            const uint16_t t = pb.pairtab[e];
            const int aa = t & 255, bb = t >> 8;
            const R v = pf[s * a.Pst + e];
            X[bb * XS + aa] = v;
            X[aa * XS + bb] = -v;
        }
        for (int i = lane; i < N; i += 32) X[i * XS + i] = R(0);
        __syncwarp();
        R tau = R(0);
        for (int c = lane; c < ncorr; c += 32) tau += xc[pb.corr_off[c] + cidx[c]];
        for (int e = lane; e < pb.P; e += 32) {
            const uint16_t t = pb.pairtab[e];
            const int aa = t & 255, bb = t >> 8;
            tau += Xt[occ[aa] * M + occ[bb]] * X[bb * XS + aa];
        }
        tau = warp_sum(tau);
        const R xt = x0 + tau;                 // sum_j O_j(n) x_j with O_0 = 1

        // ---- G = F[emp, occ] A^{-1}; Xo = X[occ, occ] ----------------------
        for (int t = lane; t < E * N; t += 32) {
            const int ie = t / N, k = t % N;
            Pm[ie * GS + k] = load_F<R>(pb, emp[ie], occ[k]);
        }
        for (int t = lane; t < N * N; t += 32) {
            const int l = t / N, k = t % N;
            Xo[l * XS + k] = Xt[occ[l] * M + occ[k]];
        }
        __syncwarp();
        warp_gemm<R, 2>(E, N, N, Pm, GS, 1, X, XS, 1, G, GS, R(1), false);
        __syncwarp();
        // ---- P = X[emp, occ] - G Xo; D = P A^{-1} (dG along x) -------------
        for (int t = lane; t < E * N; t += 32) {
            const int ie = t / N, k = t % N;
            Pm[ie * GS + k] = Xt[emp[ie] * M + occ[k]];
        }
        __syncwarp();
        warp_gemm<R, 2>(E, N, N, G, GS, 1, Xo, XS, 1, Pm, GS, R(-1), true);
        __syncwarp();
        warp_gemm<R, 2>(E, N, N, Pm, GS, 1, X, XS, 1, D, GS, R(1), false);
        for (int t = lane; t < nn; t += 32) Y[t] = R(0);
        __syncwarp();
        for (int t = lane; t < E * N; t += 32) Pm[(t / N) * GS + t % N] = R(0);

        // ---- forward: y over the moves and the diagonal, summed over spin --
        for (int t = lane; t < nex; t += 32) {
            int ia, ie;
            decode_move(t, nu, eu, ed, &ia, &ie);
            const int p = occ[ia], v = emp[ie];
            R dl;
            const R rc = corr_ratio_dir<R>(pb, cidx, p, v, xc, &dl);
            rcm[t] = rc;
            const R y = rc * (G[ie * GS + ia] * (xt + dl) + D[ie * GS + ia]);
            atomicAdd(&Y[(p % ns) * ns + (v % ns)], y);
        }
        for (int i = lane; i < N; i += 32) atomicAdd(&Y[(occ[i] % ns) * (ns + 1)], xt);
        __syncwarp();
        // ---- w_mu = sum_rs R^mu_rs y_rs, z_pq = sum_mu L^mu_pq w_mu ---------
        for (int mu = 0; mu < n_mu; ++mu) {
            R acc = R(0);
            for (int k = a.Rptr[mu] + lane; k < a.Rptr[mu + 1]; k += 32) acc += Rval[k] * Y[a.Ridx[k]];
            acc = warp_sum(acc);
            if (lane == 0) w[mu] = acc;
        }
        __syncwarp();
        for (int t = lane; t < nn; t += 32) Y[t] = R(0);
        __syncwarp();
        for (int mu = 0; mu < n_mu; ++mu) {
            const R wm = w[mu];
            for (int k = a.Lptr[mu] + lane; k < a.Lptr[mu + 1]; k += 32) atomicAdd(&Y[a.Lidx[k]], Lval[k] * wm);
        }
        __syncwarp();

        // ---- backward: z over the moves ------------------------------------
        for (int c = lane; c < ncorr; c += 32) cold[c] = R(0);
        __syncwarp();
        R W = R(0);
        for (int i = lane; i < N; i += 32) W += Y[(occ[i] % ns) * (ns + 1)];
        if (lane == 0) W += c0 * xt;
        for (int t = lane; t < nex; t += 32) {
            int ia, ie;
            decode_move(t, nu, eu, ed, &ia, &ie);
            const int p = occ[ia], v = emp[ie];
            const R z = Y[(v % ns) * ns + (p % ns)];   // z_{v p}: the move p -> v
            if (z == R(0)) continue;
            const R rc = rcm[t];
            const R g = G[ie * GS + ia];
            W += z * rc * g;
            Pm[ie * GS + ia] = z * rc;
            corr_ratio_adjoint<R>(pb, cidx, p, v, (double)(z * rc * g) * sc, a.Hx + 1, cold);
        }
        W = warp_sum(W);
        __syncwarp();
        // B = Cbar A^{-T}; G^T B
        warp_gemm<R, 2>(E, N, N, Pm, GS, 1, X, 1, XS, D, GS, R(1), false);
        __syncwarp();
        warp_gemm<R, 2>(N, N, E, G, 1, GS, D, GS, 1, Xo, XS, R(1), false);
        __syncwarp();

        // ---- scatter ------------------------------------------------------
        if (lane == 0) {
            atomicAdd(a.Hx, (double)W * sc);
            if (a.Sx) atomicAdd(a.Sx, (double)xt * sc);
        }
        for (int c = lane; c < ncorr; c += 32) {
            const int64_t k = pb.corr_off[c] + cidx[c];
            const double ic = 1.0 / __ldg(pb.C64 + k);
            atomicAdd(a.Hx + 1 + k, ((double)W * sc - (double)cold[c]) * ic);
            if (a.Sx) atomicAdd(a.Sx + 1 + k, (double)xt * ic * sc);
        }
        for (int e = lane; e < pb.P; e += 32) {
            const uint16_t t = pb.pairtab[e];
            const int aa = t & 255, bb = t >> 8;
            const int64_t idx = pb.rowbase[occ[aa]] + occ[bb];
            const R xba = X[bb * XS + aa];
            atomicAdd(Hf + idx, (double)(W * xba - Xo[aa * XS + bb] + Xo[bb * XS + aa]) * sc);
            if (a.Sx) atomicAdd(a.Sx + 1 + pb.ncp + idx, (double)(xt * xba) * sc);
        }
        for (int t = lane; t < E * N; t += 32) {
            const int ie = t / N, k = t % N;
            const R b = D[ie * GS + k];
            if (b == R(0)) continue;
            const int v = emp[ie], o = occ[k];
            if (v < o) atomicAdd(Hf + pb.rowbase[v] + o, (double)b * sc);
            else atomicAdd(Hf + pb.rowbase[o] + v, -(double)b * sc);
        }
        __syncwarp();
    }
}

// diag of S over the basis (without its 0 entry, which is 1): the mean of
// O_k(n)^2 over the samples, one warp per sample
template <typename R>
__global__ void k_lm_diag(LmArgs a, double* d) {
    const DevProblem& pb = a.pb;
    const int lane = threadIdx.x & 31;
    const R* pf = (const R*)a.pf;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t s = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < a.n_s; s += nwarps) {
        for (int c = lane; c < pb.ncorr; c += 32) {
            const int64_t k = pb.corr_off[c] + a.s_cidx[s * a.ncst + c];
            const double ic = 1.0 / __ldg(pb.C64 + k);
            atomicAdd(d + 1 + k, ic * ic * a.inv_n);
        }
        for (int e = lane; e < pb.P; e += 32) {
            const uint16_t t = pb.pairtab[e];
            const int p = a.s_occ[s * a.Nst + (t & 255)], q = a.s_occ[s * a.Nst + (t >> 8)];
            const double v = (double)pf[s * a.Pst + e];
            atomicAdd(d + 1 + pb.ncp + pb.rowbase[p] + q, v * v * a.inv_n);
        }
    }
}

// part[b * k + j] = partial sums of V[:, j] . u over block b's slice
__global__ void __launch_bounds__(256) k_lm_dots(const double* V, int64_t ld, int k, const double* u, int64_t n,
                                                 double* part) {
    __shared__ double red[8];
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per, i1 = min(n, i0 + per);
    for (int j = 0; j < k; ++j) {
        double acc = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += V[(int64_t)j * ld + i] * u[i];
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            part[(int64_t)blockIdx.x * k + j] = t;
        }
        __syncthreads();
    }
}

// out[j] = sum over blocks of part[b * k + j]
__global__ void k_lm_dots_reduce(const double* part, int nb, int k, double* out) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[(int64_t)b * k + j];
        out[j] = t;
    }
}

// out = alpha out + sum_j c[j] V[:, j]
__global__ void __launch_bounds__(256) k_lm_combine(double* out, const double* V, int64_t ld, int k, const double* c,
                                                    int64_t n, double alpha) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = alpha == 0.0 ? 0.0 : alpha * out[i];
        for (int j = 0; j < k; ++j) acc += c[j] * V[(int64_t)j * ld + i];
        out[i] = acc;
    }
}

// t = -r / (d + eps D), D = diag(0, 1, .., 1)
__global__ void __launch_bounds__(256) k_lm_precond(double* t, const double* r, const double* d, double eps, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = -r[i] / (d[i] + (i > 0 ? eps : 0.0));
}

// alpha += x_{1:} / Sx0 (Sec. II.B: the update relative to the component of
// the new state along Psi in the basis orthogonalised to Psi)
__global__ void __launch_bounds__(256) k_lm_update(UpdateArgs a, const double* x, double scale) {
    const int64_t nv = a.ncp + a.npf;
    int bad = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (int64_t)gridDim.x * blockDim.x) {
        const double d = scale * x[1 + k];
        if (k < a.ncp) {
            const double c = a.C64[k] + d;
            if (c == 0.0) bad |= ST_SINGULAR;
            if (!isfinite(c)) bad |= ST_NONFINITE;
            a.C64[k] = c;
            a.C32[k] = (float)c;
            a.invC64[k] = 1.0 / c;
            a.invC32[k] = (float)(1.0 / c);
        } else {
            const uint32_t pq = a.pq_of[k - a.ncp];
            const int p = (int)(pq & 0xFFFFu), q = (int)(pq >> 16);
            const double f = a.F64[(int64_t)p * a.M + q] + d;
            if (!isfinite(f)) bad |= ST_NONFINITE;
            a.F64[(int64_t)p * a.M + q] = f;
            a.F64[(int64_t)q * a.M + p] = -f;
            a.F32[(int64_t)p * a.M + q] = (float)f;
            a.F32[(int64_t)q * a.M + p] = -(float)f;
        }
    }
    if (bad) atomicOr(a.status, bad);
}

template __global__ void k_lm_diag<double>(LmArgs, double*);
template __global__ void k_lm_diag<float>(LmArgs, double*);
template __global__ void k_lm_prep<double>(DevProblem, const double*, double*, double*);
template __global__ void k_lm_prep<float>(DevProblem, const double*, float*, float*);
template __global__ void k_lm_apply<double>(LmArgs);
template __global__ void k_lm_apply<float>(LmArgs);

}  // namespace vmc
