// fit_eigen.cu -- scatter matrices and the generalized eigensolve, on one CTA.
//
// Section 2 of the paper computes the within-class and between-class
// covariance matrices of the training pixels and takes the eigenvectors of
// their eigenanalysis as the canonical vectors; Section 4 solves that
// eigenanalysis with GSL's generalized symmetric-definite solver, i.e.
//     Sb v = lambda Sw v .
// Everything here runs in FP64 on a single CTA, so the eigensolve never
// touches the host:
//
//  1. Sw and Sb from the exact integer moments of fit_moments.cu:
//       Sw[i][j] = sum_c (n_c M_c[i][j] - s_c[i] s_c[j]) / n_c
//     whose numerator is an exact 128-bit integer, and Sb = Mb Mb^T with the
//     B x K matrix Mb[:, c] = sqrt(n_c) (mu_c - mu), whose entries are
//     exact 128-bit numerators over n_c N;
//  2. Cholesky Sw = L L^T (right-looking), carrying Mb along as extra
//     columns so the same elimination yields G = L^-1 Mb;
//  3. L^-1 Sb L^-T = G G^T has rank <= K - 1 and the same non-zero
//     eigenvalues as the K x K matrix G^T G, which is diagonalized by the
//     cyclic Jacobi method in round-robin (parallel) order; the rotation
//     angle is taken in FP32 and the rotation itself made orthogonal to
//     FP64 accuracy by a Newton step on its cosine;
//  4. u_j = G w_j / sqrt(lambda_j) are the eigenvectors of G G^T with
//     non-zero eigenvalue; the eigenvalue-0 directions (not unique) are
//     completed by pivoted Gram-Schmidt on the unit vectors, applied twice;
//  5. V = L^-T U (so V^T Sw V = I), the sign convention (largest-magnitude
//     component positive, lowest band on a tie), and the FP32 coefficients
//     used by the projection kernels.
#include <math.h>

#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int MAX_SWEEPS = 60;
constexpr double OFF_TOL2 = 1e-28;  // squared off-diagonal norm of the unit-norm K x K matrix

struct FinSmem {
    double A[MAXB][MAXB + MAXK + 1];  // [Sw | Mb] during elimination, then back-substitution work
    double L[MAXB][MAXB + 1];
    double G[MAXB][MAXK + 1];
    double T[MAXK][MAXK + 1];
    double Wv[MAXK][MAXK + 1];
    double U[MAXB][MAXB + 1];
    double V[MAXB][MAXB + 1];
    double swd[MAXB];
    double invd[MAXB];
    double lam[MAXB];
    double res[MAXB];
    double q[MAXB];
    double cvec[MAXB];
    double rot_c[MAXK / 2], rot_s[MAXK / 2];
    int rot_p[MAXK / 2], rot_q[MAXK / 2], rot_ok[MAXK / 2];
    int order[MAXK];
    unsigned long long n[MAXK];
    unsigned long long tot[MAXB];
    unsigned long long N;
    double fro;
    int fail;
    int r_eff;
    int pivot;
};

__device__ inline unsigned long long mom_get(const DevModel* dm, const MomShape& sh, int c, int i, int j)
{
    if (i > j) { const int t = i; i = j; j = t; }
    return dm->mom[c][blk_index(i >> 2, j >> 2, sh.nb)][(i & 3) * 4 + (j & 3)];
}

__device__ inline double i128_to_double(__int128 v)
{
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
    const double d = static_cast<double>(static_cast<unsigned long long>(u >> 64)) * 18446744073709551616.0 +
                     static_cast<double>(static_cast<unsigned long long>(u));
    return neg ? -d : d;
}

// 1 / sqrt(d) in FP64: an FP32 estimate refined by two Newton steps on
// f(r) = 1 / r^2 - d (each step squares the relative error: ~1e-7 -> ~1e-14
// -> rounding level).
__device__ inline double rsqrt_fp64(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double r = static_cast<double>(rsqrtf(static_cast<float>(d)));
    double e = fma(-d * r, r, 1.0);
    r = fma(0.5 * r, e, r);
    e = fma(-d * r, r, 1.0);
    r = fma(0.5 * r, e, r);
    return r;
}

__device__ inline double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Player at seat i in round `round` of a round-robin tournament of n (even)
// players: seat 0 stays, the others rotate.  Seats i and n-1-i meet.
__device__ inline int rr_player(int i, int round, int n)
{
    return i == 0 ? 0 : 1 + (i - 1 + round) % (n - 1);
}

// Complete U[:, j0 .. j1) to an orthonormal set with pivoted Gram-Schmidt:
// each new column is the unit vector with the largest residual against the
// columns so far (lowest index on ties), orthogonalized twice.
__device__ void complete_basis(FinSmem& sm, int B, int j0, int j1)
{
    const int tid = threadIdx.x;
    for (int j = j0; j < j1; ++j) {
        if (tid < B) {
            double s = 0.0;
            for (int l = 0; l < j; ++l) s += sm.U[tid][l] * sm.U[tid][l];
            sm.res[tid] = 1.0 - s;
        }
        __syncthreads();
        if (tid == 0) {
            int best = 0;
            for (int i = 1; i < B; ++i)
                if (sm.res[i] > sm.res[best]) best = i;
            sm.pivot = best;
        }
        __syncthreads();
        const int piv = sm.pivot;
        if (tid < B) {
            double s = (tid == piv) ? 1.0 : 0.0;
            for (int l = 0; l < j; ++l) s -= sm.U[piv][l] * sm.U[tid][l];
            sm.q[tid] = s;
        }
        __syncthreads();
        if (tid < j) {
            double s = 0.0;
            for (int b = 0; b < B; ++b) s += sm.U[b][tid] * sm.q[b];
            sm.cvec[tid] = s;
        }
        __syncthreads();
        if (tid < B) {
            double s = sm.q[tid];
            for (int l = 0; l < j; ++l) s -= sm.cvec[l] * sm.U[tid][l];
            sm.q[tid] = s;
        }
        __syncthreads();
        if (tid < 32) {
            double s = 0.0;
            for (int b = tid; b < B; b += 32) s += sm.q[b] * sm.q[b];
            s = warp_sum(s);
            if (tid == 0) sm.res[0] = rsqrt_fp64(s);
        }
        __syncthreads();
        const double inv = sm.res[0];
        if (tid < B) sm.U[tid][j] = sm.q[tid] * inv;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TPB) k_fit_finalize(DevModel* __restrict__ dm, int B, int K, int nvec)
{
    extern __shared__ __align__(16) unsigned char fin_dyn[];
    FinSmem& sm = *reinterpret_cast<FinSmem*>(fin_dyn);
    const MomShape sh = mom_shape(B);
    const int tid = threadIdx.x;
    if (dm->status != 0) return;  // the moments pass already failed

    // ---- 1. counts, totals, Sw and Mb (exact numerators) -------------------
    if (tid < K) sm.n[tid] = mom_get(dm, sh, tid, B, B);
    if (tid < B) {
        unsigned long long t = 0;
        for (int c = 0; c < K; ++c) t += mom_get(dm, sh, c, tid, B);
        sm.tot[tid] = t;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long N = 0;
        int fail = 0;
        for (int c = 0; c < K; ++c) {
            N += sm.n[c];
            if (sm.n[c] == 0) fail = CVA_ERR_EMPTY_CLASS;
        }
        sm.N = N;
        sm.fail = fail;
    }
    __syncthreads();
    if (sm.fail) {
        if (tid == 0) set_status(dm, sm.fail);
        return;
    }
    for (int e = tid; e < B * B; e += TPB) {
        const int i = e / B, j = e - (e / B) * B;
        if (j < i) continue;
        double acc = 0.0;
        for (int c = 0; c < K; ++c) {
            const unsigned long long nc = sm.n[c];
            const __int128 num = static_cast<__int128>(nc) * static_cast<__int128>(mom_get(dm, sh, c, i, j)) -
                                 static_cast<__int128>(mom_get(dm, sh, c, i, B)) *
                                     static_cast<__int128>(mom_get(dm, sh, c, j, B));
            acc += i128_to_double(num) / static_cast<double>(nc);
        }
        sm.A[i][j] = acc;
        sm.A[j][i] = acc;
        dm->Sw[i][j] = acc;
        dm->Sw[j][i] = acc;
    }
    for (int e = tid; e < B * K; e += TPB) {
        const int b = e / K, c = e - (e / K) * K;
        const unsigned long long nc = sm.n[c];
        const unsigned long long s = mom_get(dm, sh, c, b, B);
        const __int128 num = static_cast<__int128>(sm.N) * static_cast<__int128>(s) -
                             static_cast<__int128>(nc) * static_cast<__int128>(sm.tot[b]);
        const double diff = i128_to_double(num) / (static_cast<double>(nc) * static_cast<double>(sm.N));
        sm.A[b][B + c] = sqrt(static_cast<double>(nc)) * diff;
        dm->mu_c[c][b] = static_cast<double>(s) / static_cast<double>(nc);
    }
    if (tid < B) dm->mu[tid] = static_cast<double>(sm.tot[tid]) / static_cast<double>(sm.N);
    if (tid < K) dm->n[tid] = static_cast<long long>(sm.n[tid]);
    __syncthreads();
    for (int e = tid; e < B * B; e += TPB) {
        const int i = e / B, j = e - (e / B) * B;
        double acc = 0.0;
        for (int c = 0; c < K; ++c) acc += sm.A[i][B + c] * sm.A[j][B + c];
        dm->Sb[i][j] = acc;
    }
    if (tid < B) sm.swd[tid] = sm.A[tid][tid];
    for (int e = tid; e < MAXB * (MAXB + 1); e += TPB) (&sm.L[0][0])[e] = 0.0;
    __syncthreads();

    // ---- 2. Cholesky of Sw with Mb carried along: L and G = L^-1 Mb ---------
    for (int j = 0; j < B; ++j) {
        if (tid == 0) {
            const double d = sm.A[j][j];
            if (!(d > PIVOT_REL * sm.swd[j])) {
                sm.fail = CVA_ERR_NOT_SPD;
            } else {
                const double r = rsqrt_fp64(d);
                sm.invd[j] = r;
                sm.L[j][j] = d * r;
            }
        }
        __syncthreads();
        if (sm.fail) break;
        const double r = sm.invd[j];
        const double r2 = r * r;
        const int m = B - j - 1;
        const int na = m, nbk = K, nc = m * m, nd = m * K;
        for (int e = tid; e < na + nbk + nc + nd; e += TPB) {
            if (e < na) {
                const int i = j + 1 + e;
                sm.L[i][j] = sm.A[i][j] * r;
            } else if (e < na + nbk) {
                const int c = e - na;
                sm.G[j][c] = sm.A[j][B + c] * r;
            } else if (e < na + nbk + nc) {
                const int q = e - na - nbk;
                const int i = j + 1 + q / m, l = j + 1 + q % m;
                if (l <= i) sm.A[i][l] -= sm.A[i][j] * sm.A[l][j] * r2;
            } else {
                const int q = e - na - nbk - nc;
                const int i = j + 1 + q / K, c = q % K;
                sm.A[i][B + c] -= sm.A[i][j] * sm.A[j][B + c] * r2;
            }
        }
        __syncthreads();
    }
    if (sm.fail) {
        if (tid == 0) set_status(dm, sm.fail);
        return;
    }
    for (int e = tid; e < B * B; e += TPB) {
        const int i = e / B, j = e - (e / B) * B;
        dm->L[i][j] = sm.L[i][j];
    }
    if (tid < B) dm->Linvd[tid] = sm.invd[tid];

    // ---- 3. T = G^T G scaled to unit Frobenius norm, then Jacobi -------------
    for (int e = tid; e < K * K; e += TPB) {
        const int a = e / K, b = e - (e / K) * K;
        double s = 0.0;
        for (int i = 0; i < B; ++i) s += sm.G[i][a] * sm.G[i][b];
        sm.T[a][b] = s;
    }
    __syncthreads();
    if (tid < 32) {
        double s = 0.0;
        for (int e = tid; e < K * K; e += 32) s += sm.T[e / K][e % K] * sm.T[e / K][e % K];
        s = warp_sum(s);
        if (tid == 0) sm.fro = sqrt(s);
    }
    __syncthreads();
    const double fro = sm.fro;
    if (fro > 0.0) {
        const double inv = 1.0 / fro;
        for (int e = tid; e < K * K; e += TPB) sm.T[e / K][e % K] *= inv;
    }
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        for (int e = lane; e < K * K; e += 32) sm.Wv[e / K][e % K] = (e / K == e % K) ? 1.0 : 0.0;
        __syncwarp();
        const int n = K + (K & 1), half = n / 2;
        bool converged = false;
        for (int sweep = 0; sweep <= MAX_SWEEPS; ++sweep) {
            double off = 0.0;
            for (int e = lane; e < K * K; e += 32) {
                const int a = e / K, b = e % K;
                if (a != b) off += sm.T[a][b] * sm.T[a][b];
            }
            off = warp_sum(off);
            if (off <= OFF_TOL2) { converged = true; break; }
            if (sweep == MAX_SWEEPS) break;
            for (int round = 0; round < n - 1; ++round) {
                if (lane < half) {
                    const int a = rr_player(lane, round, n), b = rr_player(n - 1 - lane, round, n);
                    const int p = min(a, b), q = max(a, b);
                    int ok = 0;
                    double cs = 1.0, sn = 0.0;
                    if (q < K) {
                        const float apq = static_cast<float>(sm.T[p][q]);
                        if (apq != 0.0f) {
                            const float tau = static_cast<float>(sm.T[q][q] - sm.T[p][p]) / (2.0f * apq);
                            float t;
                            if (fabsf(tau) > 1e15f) t = 0.5f / tau;
                            else t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
                            const double td = static_cast<double>(t);
                            cs = rsqrt_fp64(fma(td, td, 1.0));
                            sn = td * cs;
                            ok = 1;
                        }
                    }
                    sm.rot_p[lane] = p;
                    sm.rot_q[lane] = q;
                    sm.rot_c[lane] = cs;
                    sm.rot_s[lane] = sn;
                    sm.rot_ok[lane] = ok;
                }
                __syncwarp();
                for (int e = lane; e < K * half; e += 32) {  // T <- T J (columns p, q)
                    const int r = e % K, w = e / K;
                    if (!sm.rot_ok[w]) continue;
                    const int p = sm.rot_p[w], q = sm.rot_q[w];
                    const double cs = sm.rot_c[w], sn = sm.rot_s[w];
                    const double a = sm.T[r][p], b = sm.T[r][q];
                    sm.T[r][p] = cs * a - sn * b;
                    sm.T[r][q] = sn * a + cs * b;
                }
                __syncwarp();
                for (int e = lane; e < K * half; e += 32) {  // T <- J^T T (rows), W <- W J
                    const int r = e % K, w = e / K;
                    if (!sm.rot_ok[w]) continue;
                    const int p = sm.rot_p[w], q = sm.rot_q[w];
                    const double cs = sm.rot_c[w], sn = sm.rot_s[w];
                    const double a = sm.T[p][r], b = sm.T[q][r];
                    sm.T[p][r] = cs * a - sn * b;
                    sm.T[q][r] = sn * a + cs * b;
                    const double wa = sm.Wv[r][p], wb = sm.Wv[r][q];
                    sm.Wv[r][p] = cs * wa - sn * wb;
                    sm.Wv[r][q] = sn * wa + cs * wb;
                }
                __syncwarp();
            }
        }
        if (lane == 0) {
            if (!converged) sm.fail = CVA_ERR_NO_CONVERGENCE;
            // eigenvalues in descending order (selection, lowest index first on ties)
            int used = 0;
            for (int j = 0; j < K; ++j) {
                int best = -1;
                for (int i = 0; i < K; ++i) {
                    if (used & (1 << i)) continue;
                    if (best < 0 || sm.T[i][i] > sm.T[best][best]) best = i;
                }
                used |= 1 << best;
                sm.order[j] = best;
            }
            const int rmax = min(K - 1, B);
            const double top = sm.T[sm.order[0]][sm.order[0]];
            int r = 0;
            while (r < rmax && top > 0.0 && sm.T[sm.order[r]][sm.order[r]] > 1e-12 * top) ++r;
            sm.r_eff = r;
            for (int j = 0; j < B; ++j) sm.lam[j] = (j < r) ? sm.T[sm.order[j]][sm.order[j]] * fro : 0.0;
        }
    }
    __syncthreads();
    if (sm.fail) {
        if (tid == 0) set_status(dm, sm.fail);
        return;
    }
    const int r = sm.r_eff;
    const int nv = nvec > B ? B : nvec;

    // ---- 4. whitened eigenvectors, completed where lambda = 0 --------------
    const int rr = r < nv ? r : nv;
    for (int e = tid; e < B * rr; e += TPB) {
        const int b = e / rr, j = e - (e / rr) * rr;
        const int w = sm.order[j];
        double s = 0.0;
        for (int c = 0; c < K; ++c) s += sm.G[b][c] * sm.Wv[c][w];
        sm.U[b][j] = s * rsqrt_fp64(sm.lam[j]);
    }
    __syncthreads();
    if (nv > r) complete_basis(sm, B, r, nv);
    const int ncols = nv;

    // ---- 5. V = L^-T U by right-looking back substitution -------------------
    for (int e = tid; e < B * ncols; e += TPB) {
        const int b = e / ncols, j = e - (e / ncols) * ncols;
        sm.A[b][j] = sm.U[b][j];
    }
    __syncthreads();
    for (int i = B - 1; i >= 0; --i) {
        if (tid < ncols) sm.V[i][tid] = sm.A[i][tid] * sm.invd[i];
        __syncthreads();
        for (int e = tid; e < i * ncols; e += TPB) {
            const int l = e / ncols, j = e - (e / ncols) * ncols;
            sm.A[l][j] -= sm.L[i][l] * sm.V[i][j];
        }
        __syncthreads();
    }

    // sign convention: largest-magnitude component positive, lowest band on ties
    if (tid < ncols) {
        const int j = tid;
        double big = 0.0;
        for (int b = 0; b < B; ++b) big = fmax(big, fabs(sm.V[b][j]));
        int arg = 0;
        for (int b = 0; b < B; ++b)
            if (fabs(sm.V[b][j]) >= big * (1.0 - TIE_REL)) { arg = b; break; }
        if (sm.V[arg][j] < 0.0)
            for (int b = 0; b < B; ++b) { sm.V[b][j] = -sm.V[b][j]; sm.U[b][j] = -sm.U[b][j]; }
    }
    __syncthreads();

    // ---- 6. publish: FP64 results, FP32 coefficients, range sentinels ------
    for (int e = tid; e < MAXB * MAXB; e += TPB) {
        const int b = e / MAXB, j = e - (e / MAXB) * MAXB;
        const bool live = b < B && j < ncols;
        dm->V[b][j] = live ? sm.V[b][j] : 0.0;
        dm->U[b][j] = live ? sm.U[b][j] : 0.0;
        dm->Vf[b][j] = live ? static_cast<float>(sm.V[b][j]) : 0.0f;
    }
    if (tid < MAXB) {
        dm->lam[tid] = tid < B ? sm.lam[tid] : 0.0;
        const double m = tid < B ? rint(dm->mu[tid]) : 0.0;
        dm->shift[tid] = MAGIC_2P23 + static_cast<float>(m);
        dm->train_range[2 * tid] = __int_as_float(0x7F800000);       // +inf
        dm->train_range[2 * tid + 1] = __int_as_float(0xFF800000);   // -inf
    }
    if (tid < ncols) {
        double s = 0.0;
        for (int b = 0; b < B; ++b) s += sm.V[b][tid] * (dm->mu[b] - rint(dm->mu[b]));
        dm->dofs[tid] = static_cast<float>(s);
    } else if (tid < MAXB) {
        dm->dofs[tid] = 0.0f;
    }
    if (tid == 0) {
        dm->r = r;
        dm->nvec = ncols;
        dm->fitted = 1;
    }
}

}  // namespace

cudaError_t launch_fit_finalize(DevModel* dm, int B, int K, int nvec, cudaStream_t s)
{
    const int smem = static_cast<int>(sizeof(FinSmem));
    cudaError_t e = cudaFuncSetAttribute(k_fit_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_fit_finalize<<<1, TPB, smem, s>>>(dm, B, K, nvec);
    return cudaGetLastError();
}

}  // namespace cva
