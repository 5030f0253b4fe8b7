// fit_eigen.cu -- scatter matrices and the generalized eigensolve, on one CTA.
//
// Section 2 of the paper computes the within-class and between-class
// covariance matrices of the training pixels and takes the eigenvectors of
// their eigenanalysis as the canonical vectors; Section 4 solves that
// eigenanalysis with GSL's generalized symmetric-definite solver, i.e.
//     Sb v = lambda Sw v .
// Everything here runs on a single CTA, so the eigensolve never touches the
// host.  Every quantity whose rounding reaches the results is carried in
// double-float arithmetic (dfloat.cuh, ~48-bit significands on the FP32
// pipe): on GB300 a dependent FP64 operation costs about 64 cycles against
// under 5 for FP32, and this kernel is one long chain of dependent steps.
// FP64 is used only to publish the results into the model.
//
//  1. Sw and Mb from the exact integer moments of fit_moments.cu:
//       Sw[i][j] = sum_c (n_c M_c[i][j] - s_c[i] s_c[j]) / n_c
//     whose numerators are exact 128-bit integers (the cancellation happens
//     before any rounding), and the B x K matrix
//       Mb[:, c] = sqrt(n_c) (mu_c - mu),  mu_c - mu = (N s_c - n_c S) / (n_c N)
//     again from exact numerators, so that Sb = Mb Mb^T;
//  2. right-looking Cholesky Sw = L L^T with Mb carried along as extra
//     columns, giving G = L^-1 Mb in the same elimination (one barrier per
//     column; warp 0 alone updates the next pivot and takes its reciprocal
//     square root, the critical path of the elimination);
//  3. L^-1 Sb L^-T = G G^T has rank <= K - 1 and the same non-zero
//     eigenvalues as the K x K matrix T = G^T G.  T is diagonalized by the
//     cyclic Jacobi method in FP32 (one thread, in registers, up to order 8;
//     round-robin order on one warp up to order 8 and over the block above),
//     and the eigenvectors are then
//     refined in double-float by the Ogita-Aishima iteration (usually one or
//     two steps, at most REFINE_STEPS) for symmetric eigendecompositions (T. Ogita, K. Aishima,
//     "Iterative refinement for symmetric eigenvalue decomposition", Japan J.
//     Indust. Appl. Math. 35, 2018), which restores full accuracy from the
//     FP32 start and tolerates its loss of orthogonality;
//  4. u_j = G w_j / sqrt(lambda_j) are the eigenvectors of G G^T with
//     non-zero eigenvalue; the eigenvalue-0 directions (not unique) are
//     completed by pivoted Gram-Schmidt on the unit vectors, applied twice;
//  5. V = L^-T U (so V^T Sw V = I) by back substitution, the sign convention
//     (largest-magnitude component positive, lowest band on a tie), and the
//     FP32 coefficients used by the projection kernels.
#include <math.h>

#include "cva_internal.cuh"
#include "dfloat.cuh"

namespace cva {

namespace {

constexpr int TPB = 384;  // 12 warps: one column of the elimination fits one pass from column 5 on
constexpr int NWARP = TPB / 32;
constexpr int JACOBI_SWEEPS = 40;
constexpr int REFINE_STEPS = 8;
constexpr int MAXTRI = MAXB * (MAXB + 1) / 2;

// Work space of the symmetric eigensolver for matrices of order <= NM.
template <int NM>
struct SymEig {
    df T[NM][NM + 1];       // the matrix, about unit norm
    df W[NM][NM + 1];       // eigenvectors (columns), refined
    df R[NM][NM + 1];
    df TW[NM][NM + 1];
    df S[NM][NM + 1];
    df E[NM][NM + 1];
    float Tf[NM][NM + 1];   // FP32 copy of T, diagonalized in place
    float Wf[NM][NM + 1];   // FP32 eigenvectors (identity on entry)
    df lam[NM];             // eigenvalues, in W's column order
    float rc[NM / 2], rs[NM / 2];
    int rp[NM / 2], rq[NM / 2], rok[NM / 2];
    unsigned char rr[NM][NM];
    float red[3][NWARP];
    float last_correction;  // size of the last refinement correction (see sym_eig)
    int rotated;            // a cluster rotation was applied in this step
};

// The refinement stops once its correction is below REFINE_DONE; one that is
// still at or above it after REFINE_STEPS steps did not converge.  After a
// correction of size e the remaining error is of order e^2 (the iteration
// converges quadratically), so a converged result is good to ~1e-12.
constexpr float REFINE_DONE = 1e-6f;
// Eigenvalues closer than this relative distance (to the smaller of the two)
// are refined as one cluster: the cluster's subspace is refined, the basis
// inside it is not resolved (its vectors are not determined to this
// precision), and no correction divides by their gap.
constexpr float CLUSTER_REL = 1e-7f;

struct FinSmem {
    df A[MAXB][2 * MAXB + MAXK + 1];  // [Sw | Mb | I] during elimination
    df G[MAXB][MAXK + 1];
    df Li[MAXB][MAXB + 1];        // L^-1 (lower triangular)
    SymEig<MAXK> eig;             // T = G^T G and its eigen-decomposition
    df U[MAXB][MAXB + 1];
    df V[MAXB][MAXB + 1];
    df mu[MAXB];
    df invd[MAXB];
    df lam[MAXB];
    df q[MAXB];
    df cvec[MAXB];
    df invn[MAXK];
    df sqn[MAXK];
    float swd[MAXB];
    float res[MAXB];
    int order[MAXK];
    unsigned long long n[MAXK];
    unsigned long long tot[MAXB];
    unsigned char tri_i[MAXTRI], tri_l[MAXTRI];
    unsigned long long N;
    df invN;
    df rnorm;
    df hv[MAXK];     // Householder vector of the deflation
    df gv[MAXB];     // G hv
    df beta;         // 2 / hv^T hv
    float scale;     // power of two bringing T to about unit Frobenius norm
    int fail;
    int r_eff;
    int pivot;
};

__device__ inline unsigned long long mom_get(const DevModel* dm, const MomShape& sh, int c, int i, int j)
{
    if (i > j) { const int t = i; i = j; j = t; }
    return dm->mom[c][blk_index(i >> 2, j >> 2, sh.nb)][(i & 3) * 4 + (j & 3)];
}

// The same entry from a shared-memory copy of classes 0 .. K-1 (class c at
// m + c nblk 16, in the model's block layout).
__device__ inline unsigned long long mom_s(const unsigned long long* m, const MomShape& sh, int c, int i, int j)
{
    if (i > j) { const int t = i; i = j; j = t; }
    return m[(c * sh.nblk + blk_index(i >> 2, j >> 2, sh.nb)) * 16 + (i & 3) * 4 + (j & 3)];
}

// Words of the finalize's shared-memory copy of the moments (every class at
// the largest band count).
constexpr int MOM_COPY_WORDS = MAXK * MAXBLK * 16;

__device__ inline float warp_sumf(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ inline df shfl_xor_df(df v, int o)
{
    return df_make(__shfl_xor_sync(0xFFFFFFFFu, v.hi, o), __shfl_xor_sync(0xFFFFFFFFu, v.lo, o));
}

__device__ inline df warp_sum_df(df v)
{
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_xor_df(v, o));
    return v;
}

// Player at seat i in round `round` of a round-robin tournament of n (even)
// players: seat 0 stays, the others rotate.  Seats i and n-1-i meet.
__device__ inline int rr_player(int i, int round, int n)
{
    return i == 0 ? 0 : 1 + (i - 1 + round) % (n - 1);
}

// Block-wide maximum of a per-thread float (slot selects the scratch row).
template <int NM>
__device__ inline float block_maxf(SymEig<NM>& e, float v, int slot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) e.red[slot][warp] = v;
    __syncthreads();
    float m = e.red[slot][0];
    for (int w = 1; w < NWARP; ++w) m = fmaxf(m, e.red[slot][w]);
    return m;
}

// Sum over the team: warp 0 (TEAM = 32) or the whole block (TEAM = TPB).
template <int NM, int TEAM>
__device__ inline float team_sumf(SymEig<NM>& e, float v)
{
    v = warp_sumf(v);
    if (TEAM == 32) return v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) e.red[0][warp] = v;
    __syncthreads();
    float t = 0.0f;
    for (int w = 0; w < NWARP; ++w) t += e.red[0][w];
    __syncthreads();  // the scratch row is free again
    return t;
}

template <int TEAM>
__device__ inline void team_sync()
{
    if (TEAM == 32) __syncwarp();
    else __syncthreads();
}

// Cyclic Jacobi on e.Tf (round-robin order) in FP32, accumulating the
// rotations in e.Wf.  Run by warp 0 alone (TEAM = 32) for orders 5 to 8 or by
// the whole block (TEAM = TPB) above, which applies the rotations of a round
// in parallel over all its threads; jacobi_serial takes the orders below.
template <int NM, int TEAM>
__device__ void jacobi_team(SymEig<NM>& e, int n)
{
    const int me = TEAM == 32 ? static_cast<int>(threadIdx.x & 31) : static_cast<int>(threadIdx.x);
    const int m = n + (n & 1), half = m / 2;
    for (int q = me; q < (m - 1) * m; q += TEAM) {  // round-robin seating, one row per round
        const int round = q / m, seat = q - (q / m) * m;
        e.rr[round][seat] = static_cast<unsigned char>(rr_player(seat, round, m));
    }
    float tot = 0.0f;
    for (int q = me; q < n * n; q += TEAM) tot = fmaf(e.Tf[q / n][q % n], e.Tf[q / n][q % n], tot);
    tot = team_sumf<NM, TEAM>(e, tot);
    team_sync<TEAM>();
    float prev = 3.0e38f;
    for (int sweep = 0; sweep < JACOBI_SWEEPS; ++sweep) {
        float off = 0.0f;
        for (int q = me; q < n * n; q += TEAM) {
            const int a = q / n, b = q % n;
            if (a != b) off = fmaf(e.Tf[a][b], e.Tf[a][b], off);
        }
        off = team_sumf<NM, TEAM>(e, off);
        // converged, or stalled at FP32 rounding; the stall is only judged once
        // the off-diagonal part is small, as an early sweep may shrink it by
        // less than a factor of 4
        if (off <= 1e-11f * tot || (off >= 0.25f * prev && off <= 1e-9f * tot)) break;
        prev = off;
        for (int round = 0; round < m - 1; ++round) {
            if (me < half) {
                const int a = e.rr[round][me], b = e.rr[round][m - 1 - me];
                const int p = min(a, b), q = max(a, b);
                int ok = 0;
                float cs = 1.0f, sn = 0.0f;
                if (q < n) {
                    const float apq = e.Tf[p][q];
                    if (apq != 0.0f) {
                        // approximate intrinsics suffice: the refinement below
                        // restores accuracy, only orthogonal-enough rotations matter
                        const float tau = __fdividef(e.Tf[q][q] - e.Tf[p][p], 2.0f * apq);
                        float t;
                        if (fabsf(tau) > 1e15f) t = __fdividef(0.5f, tau);
                        else {
                            const float q = fmaf(tau, tau, 1.0f);  // >= 1: q rsqrt(q) is sqrt(q)
                            t = copysignf(__fdividef(1.0f, fabsf(tau) + q * rsqrtf(q)), tau);
                        }
                        cs = rsqrtf(fmaf(t, t, 1.0f));
                        sn = t * cs;
                        ok = 1;
                    }
                }
                e.rp[me] = p;
                e.rq[me] = q;
                e.rc[me] = cs;
                e.rs[me] = sn;
                e.rok[me] = ok;
            }
            team_sync<TEAM>();
            for (int q = me; q < n * half; q += TEAM) {  // T <- T J
                const int r = q % n, w = q / n;
                if (!e.rok[w]) continue;
                const int p = e.rp[w], qq = e.rq[w];
                const float cs = e.rc[w], sn = e.rs[w];
                const float a = e.Tf[r][p], b = e.Tf[r][qq];
                e.Tf[r][p] = cs * a - sn * b;
                e.Tf[r][qq] = sn * a + cs * b;
            }
            team_sync<TEAM>();
            for (int q = me; q < n * half; q += TEAM) {  // T <- J^T T, W <- W J
                const int r = q % n, w = q / n;
                if (!e.rok[w]) continue;
                const int p = e.rp[w], qq = e.rq[w];
                const float cs = e.rc[w], sn = e.rs[w];
                const float a = e.Tf[p][r], b = e.Tf[qq][r];
                e.Tf[p][r] = cs * a - sn * b;
                e.Tf[qq][r] = sn * a + cs * b;
                const float wa = e.Wf[r][p], wb = e.Wf[r][qq];
                e.Wf[r][p] = cs * wa - sn * wb;
                e.Wf[r][qq] = sn * wa + cs * wb;
            }
            team_sync<TEAM>();
        }
    }
}

// The same cyclic Jacobi method for orders N <= 4 on one thread, with the
// matrix and the accumulated rotations in registers and the rotations taken
// in row-cyclic order: at these orders a warp spends most of each round on
// shared-memory round trips and warp barriers, which a single thread avoids.
// The fit kernels (one page, and one CTA a page in the batched form) take it
// up to order 8.  They then need 155 registers, one CTA an SM (a batch of
// more pages than SMs runs its eigensolves in two waves); capped at order 4
// they needed 56 and took longer (ncu on the 4-class benchmark fit: 46-48 us
// against 42 us; the order-5 Jacobi on warp 0 was slower still).
template <int N, int NM>
__device__ void jacobi_serial(SymEig<NM>& e)
{
    float a[N][N], w[N][N];
    float tot = 0.0f;
    #pragma unroll
    for (int i = 0; i < N; ++i)
        #pragma unroll
        for (int j = 0; j < N; ++j) {
            a[i][j] = e.Tf[i][j];
            w[i][j] = (i == j) ? 1.0f : 0.0f;
            tot = fmaf(a[i][j], a[i][j], tot);
        }
    float prev = 3.0e38f;
    #pragma unroll 1
    for (int sweep = 0; sweep < JACOBI_SWEEPS; ++sweep) {
        float off = 0.0f;
        #pragma unroll
        for (int i = 0; i < N; ++i)
            #pragma unroll
            for (int j = 0; j < N; ++j)
                if (i != j) off = fmaf(a[i][j], a[i][j], off);
        // converged, or stalled at FP32 rounding (judged as in jacobi_team)
        if (off <= 1e-11f * tot || (off >= 0.25f * prev && off <= 1e-9f * tot)) break;
        prev = off;
        #pragma unroll
        for (int p = 0; p < N - 1; ++p)
            #pragma unroll
            for (int q = p + 1; q < N; ++q) {
                const float apq = a[p][q];
                if (apq == 0.0f) continue;
                // approximate intrinsics suffice: the refinement restores accuracy
                const float tau = __fdividef(a[q][q] - a[p][p], 2.0f * apq);
                float t;
                if (fabsf(tau) > 1e15f) t = __fdividef(0.5f, tau);
                else {
                    const float u = fmaf(tau, tau, 1.0f);  // >= 1: u rsqrt(u) is sqrt(u)
                    t = copysignf(__fdividef(1.0f, fabsf(tau) + u * rsqrtf(u)), tau);
                }
                const float cs = rsqrtf(fmaf(t, t, 1.0f));
                const float sn = t * cs;
                #pragma unroll
                for (int k = 0; k < N; ++k) {  // A <- A J
                    const float x = a[k][p], y = a[k][q];
                    a[k][p] = cs * x - sn * y;
                    a[k][q] = sn * x + cs * y;
                }
                #pragma unroll
                for (int k = 0; k < N; ++k) {  // A <- J^T A, W <- W J
                    const float x = a[p][k], y = a[q][k];
                    a[p][k] = cs * x - sn * y;
                    a[q][k] = sn * x + cs * y;
                    const float wx = w[k][p], wy = w[k][q];
                    w[k][p] = cs * wx - sn * wy;
                    w[k][q] = sn * wx + cs * wy;
                }
            }
    }
    #pragma unroll
    for (int i = 0; i < N; ++i)
        #pragma unroll
        for (int j = 0; j < N; ++j) {
            e.Tf[i][j] = a[i][j];
            e.Wf[i][j] = w[i][j];
        }
}

// Eigen-decomposition of the symmetric n x n matrix e.T (n <= NM, scaled to
// about unit norm; e.Tf holds its FP32 copy and e.Wf the identity on entry).
// The cyclic Jacobi method in FP32 runs on thread 0 for orders up to SER, on
// warp 0 up to 8 and on the whole block above; the eigenvectors are then
// refined in double-float by the Ogita-Aishima iteration for symmetric
// eigendecompositions (T. Ogita, K. Aishima, "Iterative refinement for
// symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018),
// whose matrix products are spread over the whole block.  Leaves the eigenvectors in e.W
// (columns) and the eigenvalues in e.lam, unsorted.  Every thread of the
// block calls it.
//
// The size of a correction E (W <- W (I + E)) is measured by what it changes
// in the result.  For principal components (`canonical` false) the columns of
// W are the output: the size is max |E_ab|.  For canonical variates the output
// of column b is G w_b / sqrt(lambda_b), which a correction moves by
// sum_a E_ab sqrt(lambda_a / lambda_b) (G w_a / sqrt(lambda_a)): the size is
// max |E_ab| sqrt(lambda_a / lambda_b) over columns b of non-zero eigenvalue,
// and columns of the eigenvalue-0 direction of T = G^T G (G w = 0 there, so
// no correction along it reaches a canonical vector) do not count.
//
// Clusters.  A pair whose eigenvalue estimates are closer than the
// iteration's error bound delta (absolute: about 1e-7 |T| after the FP32
// start) is refined as a cluster, and the refinement leaves the rotation
// inside it alone.  Eigenvalues far below the largest can fall into one
// cluster with each other or with the eigenvalue 0 of T even though they
// are well apart in relative terms; left alone, their vectors stay mixed at
// the FP32 start's level, which for canonical variates mixes the small
// eigenvalue with 0.  So whenever a pair of one cluster is still coupled
// (|s_ab| of W^T T W above rounding), thread 0 diagonalizes that 2 x 2 block
// by one Jacobi rotation of the two columns of W (and of T W), and the step
// starts over from the rotated W; once the couplings are at rounding level,
// delta falls and the pairs are refined individually.
template <int NM>
__device__ bool cluster_rotations(SymEig<NM>& e, int n, float delta, float lm)
{
    bool rot = false;
    #pragma unroll 1
    for (int sweep = 0; sweep < 2; ++sweep) {
        #pragma unroll 1
        for (int a = 0; a < n; ++a) {
            #pragma unroll 1
            for (int b = a + 1; b < n; ++b) {
                const float la = e.lam[a].hi, lb = e.lam[b].hi;
                const float near = CLUSTER_REL * fminf(fabsf(la), fabsf(lb));
                if (fabsf(lb - la) > fmaxf(delta, near)) continue;
                df p = df_from(0.0f), q = df_from(0.0f), r = df_from(0.0f);
                #pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    p = df_fma(p, e.W[i][a], e.TW[i][a]);
                    q = df_fma(q, e.W[i][a], e.TW[i][b]);
                    r = df_fma(r, e.W[i][b], e.TW[i][b]);
                }
                // the diagonal difference and the quotient in double-float: for a
                // (nearly) degenerate pair r - p is far below FP32 resolution
                const df d = df_sub(r, p);
                if (!(fabsf(q.hi) > fmaxf(1e-6f * fabsf(d.hi), 1e-12f * lm))) continue;
                // rotation J = [[c, s], [-s, c]] with J^T [[p, q], [q, r]] J diagonal
                const float zeta = df_div(d, df_mulf(q, 2.0f)).hi;
                const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.0f)));
                const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = t * c;
                #pragma unroll 1
                for (int i = 0; i < n; ++i) {
                    const df wa = e.W[i][a], wb = e.W[i][b];
                    e.W[i][a] = df_sub(df_mulf(wa, c), df_mulf(wb, sn));
                    e.W[i][b] = df_add(df_mulf(wa, sn), df_mulf(wb, c));
                    const df ta = e.TW[i][a], tb = e.TW[i][b];
                    e.TW[i][a] = df_sub(df_mulf(ta, c), df_mulf(tb, sn));
                    e.TW[i][b] = df_add(df_mulf(ta, sn), df_mulf(tb, c));
                }
                rot = true;
            }
        }
    }
    return rot;
}

template <int NM, int SER>
__device__ void sym_eig(SymEig<NM>& e, int n, bool canonical)
{
    const int tid = threadIdx.x;
    if (n > 8) {
        jacobi_team<NM, TPB>(e, n);
    } else if (n > SER) {
        if ((tid >> 5) == 0) jacobi_team<NM, 32>(e, n);
    } else if (tid == 0) {
        switch (n) {
            case 1: jacobi_serial<1>(e); break;
            case 2: jacobi_serial<2>(e); break;
            case 3: jacobi_serial<3>(e); break;
            case 4: jacobi_serial<4>(e); break;
            default:
                if constexpr (SER >= 8) {
                    switch (n) {
                        case 5: jacobi_serial<5>(e); break;
                        case 6: jacobi_serial<6>(e); break;
                        case 7: jacobi_serial<7>(e); break;
                        default: jacobi_serial<8>(e); break;
                    }
                }
                break;
        }
    }
    __syncthreads();

    // Ogita-Aishima refinement of the eigenvectors W of T in double-float
    const int nn = n * n;
    for (int q = tid; q < nn; q += TPB) e.W[q / n][q % n] = df_from(e.Wf[q / n][q % n]);
    __syncthreads();
    for (int it = 0; it < REFINE_STEPS; ++it) {
        for (int q = tid; q < nn; q += TPB) {
            const int a = q / n, b = q % n;
            df r = df_from(0.0f), tw = df_from(0.0f);
            #pragma unroll 1
            for (int k = 0; k < n; ++k) {
                r = df_fma(r, e.W[k][a], e.W[k][b]);     // W^T W
                tw = df_fma(tw, e.T[a][k], e.W[k][b]);   // T W
            }
            e.R[a][b] = df_sub(df_from(a == b ? 1.0f : 0.0f), r);  // I - W^T W
            e.TW[a][b] = tw;
        }
        __syncthreads();
        float so = 0.0f, lm = 0.0f, rm = 0.0f;
        for (int q = tid; q < nn; q += TPB) {
            const int a = q / n, b = q % n;
            df sv = df_from(0.0f);
            #pragma unroll 1
            for (int k = 0; k < n; ++k) sv = df_fma(sv, e.W[k][a], e.TW[k][b]);  // W^T T W
            e.S[a][b] = sv;
            if (a != b) so = fmaxf(so, fabsf(sv.hi));
            else lm = fmaxf(lm, fabsf(sv.hi));
            rm = fmaxf(rm, fabsf(e.R[a][b].hi));
        }
        so = block_maxf(e, so, 0);
        lm = block_maxf(e, lm, 1);
        rm = block_maxf(e, rm, 2);
        const float delta = 2.0f * (so + lm * rm);  // cluster threshold
        if (tid < n) {  // lambda_i = s_ii / (1 - r_ii) = s_ii (1 + r_ii + r_ii^2 + ...)
            const df r = e.R[tid][tid];
            e.lam[tid] = df_mul(e.S[tid][tid], df_add(df_from(1.0f), df_mul(r, df_add(df_from(1.0f), r))));
        }
        __syncthreads();
        if (tid == 0) {
            e.rotated = cluster_rotations(e, n, delta, lm) ? 1 : 0;
            if (e.rotated) e.last_correction = 1.0f;  // not converged if the steps end here
        }
        __syncthreads();
        if (e.rotated) continue;  // the step starts over from the rotated W
        float emax = 0.0f;
        const float lnull = 1e-12f * lm;  // eigenvalue-0 columns (the rank test of the caller)
        for (int q = tid; q < nn; q += TPB) {
            const int a = q / n, b = q % n;
            df ev;
            const df gap = df_sub(e.lam[b], e.lam[a]);
            const float la = e.lam[a].hi, lb = e.lam[b].hi;
            const float near = CLUSTER_REL * fminf(fabsf(la), fabsf(lb));
            if (a == b || fabsf(gap.hi) <= fmaxf(delta, near)) {
                ev = df_mulf(e.R[a][b], 0.5f);
            } else {
                const df num = df_fma(e.S[a][b], e.lam[b], e.R[a][b]);
                ev = df_from(num.hi / gap.hi);
            }
            e.E[a][b] = ev;
            float w = 1.0f;
            if (canonical) w = (lb > lnull) ? sqrtf(fmaxf(la, 0.0f) / lb) : 0.0f;
            emax = fmaxf(emax, fabsf(ev.hi) * w);
        }
        __syncthreads();  // E complete; the red rows are free again
        emax = block_maxf(e, emax, 0);
        for (int q = tid; q < nn; q += TPB) {
            const int a = q / n, b = q % n;
            df d = df_from(0.0f);
            #pragma unroll 1
            for (int k = 0; k < n; ++k) d = df_fma(d, e.W[a][k], e.E[k][b]);  // W E
            e.TW[a][b] = d;
        }
        __syncthreads();
        for (int q = tid; q < nn; q += TPB) e.W[q / n][q % n] = df_add(e.W[q / n][q % n], e.TW[q / n][q % n]);
        __syncthreads();
        if (tid == 0) e.last_correction = emax;
        if (emax < REFINE_DONE) break;  // the next correction would be of order 1e-12
    }
}

// Complete U[:, j0 .. j1) to an orthonormal set with pivoted Gram-Schmidt:
// each new column is the unit vector with the largest residual against the
// columns so far (lowest index on ties), orthogonalized twice.
__device__ void complete_basis(FinSmem& sm, int B, int j0, int j1)
{
    const int tid = threadIdx.x;
    for (int j = j0; j < j1; ++j) {
        if (tid < B) {
            float s = 0.0f;
            #pragma unroll 1
            for (int l = 0; l < j; ++l) s = fmaf(sm.U[tid][l].hi, sm.U[tid][l].hi, s);
            sm.res[tid] = 1.0f - s;
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
            df s = df_from((tid == piv) ? 1.0f : 0.0f);
            #pragma unroll 1
            for (int l = 0; l < j; ++l) s = df_fms(s, sm.U[piv][l], sm.U[tid][l]);
            sm.q[tid] = s;
        }
        __syncthreads();
        if (tid < j) {
            df s = df_from(0.0f);
            #pragma unroll 1
            for (int b = 0; b < B; ++b) s = df_fma(s, sm.U[b][tid], sm.q[b]);
            sm.cvec[tid] = s;
        }
        __syncthreads();
        if (tid < B) {
            df s = sm.q[tid];
            #pragma unroll 1
            for (int l = 0; l < j; ++l) s = df_fms(s, sm.cvec[l], sm.U[tid][l]);
            sm.q[tid] = s;
        }
        __syncthreads();
        if (tid < 32) {
            df s = df_from(0.0f);
            for (int b = tid; b < B; b += 32) s = df_fma(s, sm.q[b], sm.q[b]);
            s = warp_sum_df(s);
            if (tid == 0) sm.rnorm = df_rsqrt(s);
        }
        __syncthreads();
        if (tid < B) sm.U[tid][j] = df_mul(sm.q[tid], sm.rnorm);
        __syncthreads();
    }
}

template <int SER>
__device__ __forceinline__ void fit_finalize_body(FinSmem& sm, unsigned long long* __restrict__ mom, DevModel* __restrict__ dm,
                                                  int B, int K, int nvec)
{
    const MomShape sh = mom_shape(B);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (dm->status != 0) return;  // an earlier pass already failed
    // the exact moments of the K classes into shared memory, all loads at once
    // (the phases below read them many times, in dependent loops)
    for (int q = tid; q < K * sh.nblk * 16; q += TPB) {
        const int c = q / (sh.nblk * 16), r = q - c * (sh.nblk * 16);
        mom[q] = dm->mom[c][r >> 4][r & 15];
    }
    __syncthreads();

    // ---- 0. counts, totals, triangle tables ---------------------------------
    if (tid < K) sm.n[tid] = mom_s(mom, sh, tid, B, B);
    if (tid < B) {
        unsigned long long t = 0;
        #pragma unroll 1
        for (int c = 0; c < K; ++c) t += mom_s(mom, sh, c, tid, B);
        sm.tot[tid] = t;
    }
    for (int i = warp; i < MAXB; i += NWARP)
        for (int l = lane; l <= i; l += 32) {
            const int q = i * (i + 1) / 2 + l;
            sm.tri_i[q] = static_cast<unsigned char>(i);
            sm.tri_l[q] = static_cast<unsigned char>(l);
        }
    __syncthreads();
    if (tid == 0) {
        unsigned long long N = 0;
        int fail = 0;
        #pragma unroll 1
        for (int c = 0; c < K; ++c) {
            N += sm.n[c];
            if (sm.n[c] == 0) fail = CVA_ERR_EMPTY_CLASS;
        }
        sm.N = N;
        sm.fail = fail;
        if (N) sm.invN = df_rcp(df_from_u64(N));
    }
    if (tid < K && sm.n[tid]) {
        const df n = df_from_u64(sm.n[tid]);
        sm.invn[tid] = df_rcp(n);
        sm.sqn[tid] = df_mul(n, df_rsqrt(n));
    }
    __syncthreads();
    if (sm.fail) {
        if (tid == 0) set_status(dm, sm.fail);
        return;
    }

    // ---- 1. class means, Sw and Mb from exact numerators ----------------------
    for (int e = tid; e < K * B; e += TPB) {
        const int c = e / B, b = e - (e / B) * B;
        const unsigned long long s = mom_s(mom, sh, c, b, B);
        dm->mu_c[c][b] = df_to_double(df_mul(df_from_u64(s), sm.invn[c]));
        const __int128 num = static_cast<__int128>(sm.N) * s - static_cast<__int128>(sm.n[c]) * sm.tot[b];
        const df v = df_mul(df_mul(df_mul(df_from_i128(num), sm.invn[c]), sm.invN), sm.sqn[c]);
        sm.A[b][B + c] = v;
        dm->Mb[b][c] = df_to_double(v);
    }
    if (tid < B) {
        sm.mu[tid] = df_mul(df_from_u64(sm.tot[tid]), sm.invN);
        dm->mu[tid] = df_to_double(sm.mu[tid]);
    }
    if (tid < K) dm->n[tid] = static_cast<long long>(sm.n[tid]);
    for (int q = tid; q < B * (B + 1) / 2; q += TPB) {
        const int i = sm.tri_i[q], l = sm.tri_l[q];
        df acc = df_from(0.0f);
        #pragma unroll 1
        for (int c = 0; c < K; ++c) {
            const __int128 num = static_cast<__int128>(sm.n[c]) * mom_s(mom, sh, c, i, l) -
                                 static_cast<__int128>(mom_s(mom, sh, c, i, B)) * mom_s(mom, sh, c, l, B);
            acc = df_add(acc, df_mul(df_from_i128(num), sm.invn[c]));
        }
        sm.A[i][l] = acc;
        sm.A[l][i] = acc;
        const double d = df_to_double(acc);
        dm->Sw[i][l] = d;
        dm->Sw[l][i] = d;
    }
    __syncthreads();
    if (tid < B) sm.swd[tid] = sm.A[tid][tid].hi;
    for (int e = tid; e < MAXB * (MAXB + 1); e += TPB) (&sm.Li[0][0])[e] = df_from(0.0f);
    for (int e = tid; e < B * B; e += TPB) {  // identity columns: the elimination turns them into L^-1
        const int i = e / B, j = e - (e / B) * B;
        sm.A[i][B + K + j] = df_from(i == j ? 1.0f : 0.0f);
    }
    __syncthreads();

    // ---- 2. Cholesky of Sw with [Mb | I] carried along: G = L^-1 Mb, L^-1 ----
    // (L itself is never needed: only the reciprocals of its diagonal)
    if (tid == 0) {
        const df d = sm.A[0][0];
        if (!(d.hi > static_cast<float>(PIVOT_REL) * sm.swd[0]) || !(d.hi > 0.0f)) sm.fail = CVA_ERR_NOT_SPD;
        else sm.invd[0] = df_rsqrt(d);
    }
    const int KB = K + B;  // carried columns: Mb then the identity
    for (int j = 0; j < B; ++j) {
        __syncthreads();
        if (sm.fail) break;
        // row j of [G | L^-1] and the trailing update, in one phase: column j
        // of L, A[i][j] r, is formed where it is used.
        // Item 0 (the next pivot, on the critical path of the elimination) is
        // warp 0's alone, so that no warp runs both paths; the other items are
        // spread over warps 1 .. NWARP-1.
        const df r = sm.invd[j];
        const int m = B - j - 1;
        const int ntri = m * (m + 1) / 2;
        const int ncar = j + 1 + K;  // carried columns with nonzero row j: Mb and identity columns 0..j
        if (warp == 0) {
            if (lane == 0 && m > 0) {  // the next pivot is final after this update: take its reciprocal square root now
                const df a = sm.A[j + 1][j];
                const df v = df_fms(sm.A[j + 1][j + 1], df_mul(a, r), df_mul(a, r));
                sm.A[j + 1][j + 1] = v;
                if (!(v.hi > static_cast<float>(PIVOT_REL) * sm.swd[j + 1]) || !(v.hi > 0.0f)) sm.fail = CVA_ERR_NOT_SPD;
                else sm.invd[j + 1] = df_rsqrt(v);
            }
            continue;
        }
        // item 0 is the pivot's while there is one (m > 0); in the last column it is G[j][0].
        // Every item is X - (Y r)(Z r) (trailing and carried entries) or Y r (row j
        // of [G | L^-1]); only the operand addresses depend on the kind, so a warp
        // whose items straddle two kinds diverges only while loading.
        const float rnc = __frcp_rn(static_cast<float>(ncar));  // (q + 1/2) rnc truncates to q / ncar exactly
        const int n1 = ntri, n2 = ntri + m * ncar, n3 = n2;
        for (int e = tid - 32 + (m > 0 ? 1 : 0); e < n3 + ncar; e += TPB - 32) {
            df X = df_from(0.0f), Y, Z = df_from(0.0f);
            df* dst;
            bool fms = true;
            if (e < n1) {
                const int i = j + 1 + sm.tri_i[e], l = j + 1 + sm.tri_l[e];
                X = sm.A[i][l]; Y = sm.A[i][j]; Z = sm.A[l][j];
                dst = &sm.A[i][l];
            } else if (e < n2) {
                const int q = e - n1;
                const int qi = static_cast<int>((static_cast<float>(q) + 0.5f) * rnc);
                const int i = j + 1 + qi, col = B + (q - qi * ncar);  // Mb columns, then identity columns 0..j
                X = sm.A[i][col]; Y = sm.A[i][j]; Z = sm.A[j][col];
                dst = &sm.A[i][col];
            } else {
                const int cc = e - n3;
                Y = sm.A[j][B + cc];
                dst = (cc < K) ? &sm.G[j][cc] : &sm.Li[j][cc - K];
                fms = false;
            }
            const df yr = df_mul(Y, r);
            const df v = df_fms(X, yr, df_mul(Z, r));
            *dst = fms ? v : yr;
        }
    }
    (void)KB;
    __syncthreads();
    if (sm.fail) {
        if (tid == 0) set_status(dm, sm.fail);
        return;
    }
    // ---- 3. deflation of T's known eigenvalue-0 direction --------------------
    // G z = 0 for z_c = sqrt(n_c / N) (sum_c n_c (mu_c - mu) = 0), so T = G^T G
    // has z as an exact eigenvector of eigenvalue 0.  With the Householder
    // reflection H = I - beta v v^T, v = z + e_{K-1} (H z = -e_{K-1}), the
    // last column of G H vanishes and its first n = K - 1 columns G' carry all
    // of T's other eigenpairs: T' = G'^T G' (order K - 1) has them, and
    // eigenvectors w' of T' give G' w' = G (H w'), the same vectors G w.
    const int n = K - 1;
    if (tid < K) {
        const df z = df_mul(sm.sqn[tid], df_rsqrt(df_from_u64(sm.N)));
        sm.hv[tid] = (tid == K - 1) ? df_add(z, df_from(1.0f)) : z;
    }
    __syncthreads();
    if (tid == 0) {
        df vv = df_from(0.0f);
        #pragma unroll 1
        for (int c = 0; c < K; ++c) vv = df_fma(vv, sm.hv[c], sm.hv[c]);
        sm.beta = df_div(df_from(2.0f), vv);
    }
    if (tid < B) {
        df g = df_from(0.0f);
        #pragma unroll 1
        for (int c = 0; c < K; ++c) g = df_fma(g, sm.G[tid][c], sm.hv[c]);
        sm.gv[tid] = g;
    }
    __syncthreads();
    for (int e = tid; e < B * n; e += TPB) {
        const int b = e / n, j = e - (e / n) * n;
        sm.G[b][j] = df_fms(sm.G[b][j], df_mul(sm.beta, sm.gv[b]), sm.hv[j]);
    }
    __syncthreads();

    // ---- 3b. T' = G'^T G', scaled by a power of two to about unit norm -------
    {
        const int KK = n * n;
        int per = 1;
        while (per * 2 * KK <= TPB && per < 32) per *= 2;
        const int e = tid / per, sub = tid - (tid / per) * per;
        df s = df_from(0.0f);
        if (e < KK) {
            const int a = e / n, b = e - (e / n) * n;
            for (int i = sub; i < B; i += per) s = df_fma(s, sm.G[i][a], sm.G[i][b]);
        }
        for (int o = per / 2; o > 0; o >>= 1) s = df_add(s, shfl_xor_df(s, o));
        if (e < KK && sub == 0) sm.eig.T[e / n][e % n] = s;
    }
    __syncthreads();
    if (tid < 32) {
        float f = 0.0f;
        for (int e = tid; e < n * n; e += 32) f = fmaf(sm.eig.T[e / n][e % n].hi, sm.eig.T[e / n][e % n].hi, f);
        f = warp_sumf(f);
        if (tid == 0) {
            int ex = 0;
            if (f > 0.0f) frexpf(sqrtf(f), &ex);
            sm.scale = pow2f(-ex);
        }
    }
    __syncthreads();
    const float scale = sm.scale;
    if (tid < n * n) {
        const int a = tid / n, b = tid % n;
        sm.eig.T[a][b] = df_mulf(sm.eig.T[a][b], scale);  // exact: a power of two
        sm.eig.Tf[a][b] = sm.eig.T[a][b].hi;
        sm.eig.Wf[a][b] = (a == b) ? 1.0f : 0.0f;
    }
    __syncthreads();

    // ---- 4. FP32 cyclic Jacobi on T', then 5. refinement ---------------------
    if (n == 1) {  // two classes: T' is 1 x 1
        if (tid == 0) {
            sm.eig.W[0][0] = df_from(1.0f);
            sm.eig.lam[0] = sm.eig.T[0][0];
            sm.eig.last_correction = 0.0f;
        }
        __syncthreads();
    } else {
        sym_eig<MAXK, SER>(sm.eig, n, true);
        __syncthreads();
    }
    if (!(sm.eig.last_correction < REFINE_DONE)) {
        if (tid == 0) set_status(dm, CVA_ERR_NO_CONVERGENCE);
        return;
    }

    // ---- 6. eigenvalues in descending order, whitened eigenvectors ----------
    if (tid == 0) {
        int used = 0;
        for (int j = 0; j < n; ++j) {
            int best = -1;
            for (int i = 0; i < n; ++i) {
                if (used & (1 << i)) continue;
                if (best < 0 || df_gt(sm.eig.lam[i], sm.eig.lam[best])) best = i;
            }
            used |= 1 << best;
            sm.order[j] = best;
        }
        const int rmax = min(K - 1, B);
        const float top = sm.eig.lam[sm.order[0]].hi;
        int r = 0;
        while (r < rmax && top > 0.0f && sm.eig.lam[sm.order[r]].hi > 1e-12f * top) ++r;
        sm.r_eff = r;
    }
    __syncthreads();
    const int r = sm.r_eff;
    const int nv = nvec > B ? B : nvec;
    const int rr = r < nv ? r : nv;
    // g_j = G w_j for the r non-zero eigenpairs; lambda_j = |g_j|^2 (the
    // Rayleigh quotient of T at w_j, formed from G: T's own rounding, of
    // order 1e-14 |T|, would limit the relative accuracy of eigenvalues far
    // below the largest) and u_j = g_j / |g_j|
    for (int e = tid; e < B * r; e += TPB) {
        const int b = e / r, j = e - (e / r) * r;
        const int w = sm.order[j];
        df s = df_from(0.0f);
        #pragma unroll 1
        for (int c = 0; c < n; ++c) s = df_fma(s, sm.G[b][c], sm.eig.W[c][w]);
        sm.U[b][j] = s;
    }
    __syncthreads();
    for (int j = warp; j < MAXB; j += NWARP) {
        df s = df_from(0.0f);
        if (j < r && lane < B) s = df_mul(sm.U[lane][j], sm.U[lane][j]);
        if (j < r) s = warp_sum_df(s);
        if (lane == 0) {
            sm.lam[j] = j < r ? s : df_from(0.0f);
            if (j < r) sm.q[j] = df_rsqrt(s);
        }
    }
    __syncthreads();
    for (int e = tid; e < B * rr; e += TPB) {
        const int b = e / rr, j = e - (e / rr) * rr;
        sm.U[b][j] = df_mul(sm.U[b][j], sm.q[j]);
    }
    __syncthreads();
    if (nv > r) complete_basis(sm, B, r, nv);
    const int ncols = nv;

    // ---- 7. V = L^-T U: each entry a split dot product over 8 lanes ---------
    {
        // the loop bound is a multiple of the block size, so every lane of a
        // warp takes part in every shuffle
        const int total = B * ncols * 8;
        const int bound = (total + TPB - 1) / TPB * TPB;
        for (int e = tid; e < bound; e += TPB) {
            const bool live = e < total;
            const int o = live ? (e >> 3) : 0, part = e & 7;
            const int b = o / ncols, j = o - (o / ncols) * ncols;
            df s8 = df_from(0.0f);
            if (live)
                for (int i = b + part; i < B; i += 8) s8 = df_fma(s8, sm.Li[i][b], sm.U[i][j]);  // (L^-1)^T[b][i] = Li[i][b]
            for (int o2 = 4; o2 > 0; o2 >>= 1) s8 = df_add(s8, shfl_xor_df(s8, o2));
            if (live && part == 0) sm.V[b][j] = s8;
        }
    }
    __syncthreads();

    // ---- 8. sign convention ---------------------------------------------------
    for (int j = warp; j < ncols; j += NWARP) {
        const df v = lane < B ? sm.V[lane][j] : df_from(0.0f);
        const df av = df_abs(v);
        df big = av;
        for (int o = 16; o > 0; o >>= 1) {
            const df other = shfl_xor_df(big, o);
            if (df_gt(other, big)) big = other;
        }
        const df thr = df_mul(big, df_make(1.0f, -static_cast<float>(TIE_REL)));
        const unsigned ties = __ballot_sync(0xFFFFFFFFu, lane < B && df_ge(av, thr));
        const int arg = __ffs(ties) - 1;
        const float sh_hi = __shfl_sync(0xFFFFFFFFu, v.hi, arg);
        const float sh_lo = __shfl_sync(0xFFFFFFFFu, v.lo, arg);
        const bool neg = sh_hi < 0.0f || (sh_hi == 0.0f && sh_lo < 0.0f);
        if (neg && lane < B) {
            sm.V[lane][j] = df_neg(sm.V[lane][j]);
            sm.U[lane][j] = df_neg(sm.U[lane][j]);
        }
    }
    __syncthreads();

    // ---- 9. publish: FP64 results, FP32 coefficients, range sentinels --------
    for (int e = tid; e < MAXB * MAXB; e += TPB) {
        const int b = e / MAXB, j = e - (e / MAXB) * MAXB;
        const bool live = b < B && j < ncols;
        dm->V[b][j] = live ? df_to_double(sm.V[b][j]) : 0.0;
        dm->Vf[b][j] = live ? sm.V[b][j].hi : 0.0f;
    }
    if (tid < MAXB) {
        dm->lam[tid] = tid < B ? df_to_double(sm.lam[tid]) : 0.0;
        const float m = tid < B ? rintf(sm.mu[tid].hi) : 0.0f;
        dm->shift[tid] = MAGIC_2P23 + m;
        dm->train_range[2 * tid] = __int_as_float(0x7F800000);       // +inf
        dm->train_range[2 * tid + 1] = __int_as_float(0xFF800000);   // -inf
    }
    for (int j = warp; j < MAXB; j += NWARP) {
        df s = df_from(0.0f);
        if (j < ncols && lane < B) s = df_mul(sm.V[lane][j], df_sub(sm.mu[lane], df_from(rintf(sm.mu[lane].hi))));
        if (j < ncols) s = warp_sum_df(s);
        if (lane == 0) dm->dofs[j] = j < ncols ? s.hi : 0.0f;
    }
    if (tid == 0) {
        dm->r = r;
        dm->nvec = ncols;
        dm->fitted = 1;
    }
}

__global__ void __launch_bounds__(TPB) k_fit_finalize(DevModel* __restrict__ dm, int B, int K, int nvec)
{
    extern __shared__ __align__(16) unsigned char fin_dyn[];
    fit_finalize_body<8>(*reinterpret_cast<FinSmem*>(fin_dyn),
                         reinterpret_cast<unsigned long long*>(fin_dyn + sizeof(FinSmem)), dm, B, K, nvec);
}

// Batched form: one CTA per page, all pages at once; the eigenvalues are
// also copied to the page's output when it asks for them.
__global__ void __launch_bounds__(TPB) kb_fit_finalize(const PageDev* __restrict__ pages)
{
    extern __shared__ __align__(16) unsigned char fin_dyn[];
    const PageDev& pg = pages[blockIdx.x];
    fit_finalize_body<8>(*reinterpret_cast<FinSmem*>(fin_dyn),
                         reinterpret_cast<unsigned long long*>(fin_dyn + sizeof(FinSmem)), pg.dm, pg.B, pg.K, pg.k);
    __syncthreads();
    if (pg.eigvals && threadIdx.x < pg.B && pg.dm->status == 0) pg.eigvals[threadIdx.x] = pg.dm->lam[threadIdx.x];
}

// ---------------------------------------------------------------------------
// Principal components (Section 2: subtract the mean, form the covariance
// matrix, take its eigenvectors, orthonormal).  From the exact moments of
// class 0 (k_pca_moments): N pixels, sums s, raw moments M;
//     C[i][j] = (N M[i][j] - s_i s_j) / (N (N - 1))   (sample covariance)
// with exact 128-bit numerators, then the same symmetric eigensolver (FP32
// Jacobi + double-float refinement) on the B x B matrix, eigenvalues in
// descending order, the same sign convention, and the same projection
// coefficients, so every projection entry point applies to the result.
// ---------------------------------------------------------------------------
struct PcaSmem {
    SymEig<MAXB> eig;
    df V[MAXB][MAXB + 1];
    df mu[MAXB];
    df lam[MAXB];
    int order[MAXB];
    unsigned long long N;
    float scale;
};

__global__ void __launch_bounds__(TPB) k_pca_finalize(DevModel* __restrict__ dm, int B, int nvec)
{
    extern __shared__ __align__(16) unsigned char pca_dyn[];
    PcaSmem& sm = *reinterpret_cast<PcaSmem*>(pca_dyn);
    const MomShape sh = mom_shape(B);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (dm->status != 0) return;
    if (tid == 0) sm.N = mom_get(dm, sh, 0, B, B);
    __syncthreads();
    const unsigned long long N = sm.N;
    if (N < 2) {
        if (tid == 0) set_status(dm, CVA_ERR_EMPTY_CLASS);
        return;
    }
    const df dN = df_from_u64(N);
    const df inv_nn1 = df_rcp(df_from_u64(N * (N - 1)));  // N (N - 1) < 2^62
    if (tid < B) sm.mu[tid] = df_div(df_from_u64(mom_get(dm, sh, 0, tid, B)), dN);
    for (int q = tid; q < B * B; q += TPB) {
        const int i = q / B, j = q - (q / B) * B;
        if (i > j) continue;
        const __int128 si = static_cast<__int128>(mom_get(dm, sh, 0, i, B));
        const __int128 sj = static_cast<__int128>(mom_get(dm, sh, 0, j, B));
        const __int128 num = static_cast<__int128>(N) * static_cast<__int128>(mom_get(dm, sh, 0, i, j)) - si * sj;
        const df c = df_mul(df_from_i128(num), inv_nn1);
        sm.eig.T[i][j] = c;
        sm.eig.T[j][i] = c;
    }
    __syncthreads();
    for (int q = tid; q < B * B; q += TPB) {  // covariance for the statistics getter
        const int i = q / B, j = q - (q / B) * B;
        dm->Sw[i][j] = df_to_double(sm.eig.T[i][j]);
    }
    if (warp == 0) {
        float f = 0.0f;
        for (int q = lane; q < B * B; q += 32) f = fmaf(sm.eig.T[q / B][q % B].hi, sm.eig.T[q / B][q % B].hi, f);
        f = warp_sumf(f);
        if (lane == 0) {
            int ex = 0;
            if (f > 0.0f) frexpf(sqrtf(f), &ex);
            sm.scale = pow2f(-ex);
        }
    }
    __syncthreads();
    const float scale = sm.scale;
    for (int q = tid; q < B * B; q += TPB) {
        const int a = q / B, b = q % B;
        sm.eig.T[a][b] = df_mulf(sm.eig.T[a][b], scale);  // exact: a power of two
        sm.eig.Tf[a][b] = sm.eig.T[a][b].hi;
        sm.eig.Wf[a][b] = (a == b) ? 1.0f : 0.0f;
    }
    __syncthreads();
    sym_eig<MAXB, 4>(sm.eig, B, false);
    __syncthreads();
    if (!(sm.eig.last_correction < REFINE_DONE)) {
        if (tid == 0) set_status(dm, CVA_ERR_NO_CONVERGENCE);
        return;
    }
    if (tid == 0) {
        unsigned int used = 0u;
        for (int j = 0; j < B; ++j) {
            int best = -1;
            for (int i = 0; i < B; ++i) {
                if (used & (1u << i)) continue;
                if (best < 0 || df_gt(sm.eig.lam[i], sm.eig.lam[best])) best = i;
            }
            used |= 1u << best;
            sm.order[j] = best;
        }
    }
    __syncthreads();
    const int ncols = nvec > B ? B : nvec;
    const float unscale = __frcp_rn(scale);  // a power of two: exact
    if (tid < B) sm.lam[tid] = df_mulf(sm.eig.lam[sm.order[tid]], unscale);
    for (int q = tid; q < B * ncols; q += TPB) {
        const int b = q / ncols, j = q - (q / ncols) * ncols;
        sm.V[b][j] = sm.eig.W[b][sm.order[j]];
    }
    __syncthreads();
    // sign convention: the largest-magnitude component positive, lowest band on a tie
    for (int j = warp; j < ncols; j += NWARP) {
        const df v = lane < B ? sm.V[lane][j] : df_from(0.0f);
        const df av = df_abs(v);
        df big = av;
        for (int o = 16; o > 0; o >>= 1) {
            const df other = shfl_xor_df(big, o);
            if (df_gt(other, big)) big = other;
        }
        const df thr = df_mul(big, df_make(1.0f, -static_cast<float>(TIE_REL)));
        const unsigned ties = __ballot_sync(0xFFFFFFFFu, lane < B && df_ge(av, thr));
        const int arg = __ffs(ties) - 1;
        const float sh_hi = __shfl_sync(0xFFFFFFFFu, v.hi, arg);
        const float sh_lo = __shfl_sync(0xFFFFFFFFu, v.lo, arg);
        const bool neg = sh_hi < 0.0f || (sh_hi == 0.0f && sh_lo < 0.0f);
        if (neg && lane < B) sm.V[lane][j] = df_neg(sm.V[lane][j]);
    }
    __syncthreads();
    for (int q = tid; q < MAXB * MAXB; q += TPB) {
        const int b = q / MAXB, j = q - (q / MAXB) * MAXB;
        const bool live = b < B && j < ncols;
        const double v = live ? df_to_double(sm.V[b][j]) : 0.0;
        dm->V[b][j] = v;
        dm->Vf[b][j] = live ? sm.V[b][j].hi : 0.0f;
    }
    for (int q = tid; q < MAXB * MAXK; q += TPB) dm->Mb[q / MAXK][q % MAXK] = 0.0;
    if (tid < MAXB) {
        dm->lam[tid] = tid < B ? df_to_double(sm.lam[tid]) : 0.0;
        dm->mu[tid] = tid < B ? df_to_double(sm.mu[tid]) : 0.0;
        if (tid < B) dm->mu_c[0][tid] = dm->mu[tid];
        const float m = tid < B ? rintf(sm.mu[tid].hi) : 0.0f;
        dm->shift[tid] = MAGIC_2P23 + m;
        dm->train_range[2 * tid] = __int_as_float(0x7F800000);       // +inf
        dm->train_range[2 * tid + 1] = __int_as_float(0xFF800000);   // -inf
    }
    for (int j = warp; j < MAXB; j += NWARP) {
        df s = df_from(0.0f);
        if (j < ncols && lane < B) s = df_mul(sm.V[lane][j], df_sub(sm.mu[lane], df_from(rintf(sm.mu[lane].hi))));
        if (j < ncols) s = warp_sum_df(s);
        if (lane == 0) dm->dofs[j] = j < ncols ? s.hi : 0.0f;
    }
    if (tid == 0) {
        dm->n[0] = static_cast<long long>(N);
        dm->cls_count[0] = static_cast<unsigned int>(N);
        dm->r = B;
        dm->nvec = ncols;
        dm->fitted = 1;
    }
}

// Sb = Mb Mb^T for the statistics getter (not on the fit path).
__global__ void k_scatter_sb(DevModel* __restrict__ dm, int B, int K)
{
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int i = e / B, j = e % B;
        double s = 0.0;
        #pragma unroll 1
        for (int c = 0; c < K; ++c) s = fma(dm->Mb[i][c], dm->Mb[j][c], s);
        dm->Sb[i][j] = s;
    }
}

}  // namespace

cudaError_t launch_fit_finalize(DevModel* dm, int B, int K, int nvec, cudaStream_t s)
{
    const int smem = static_cast<int>(sizeof(FinSmem) + sizeof(unsigned long long) * K * mom_shape(B).nblk * 16);
    cudaError_t e = cudaFuncSetAttribute(k_fit_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_fit_finalize<<<1, TPB, smem, s>>>(dm, B, K, nvec);
    return cudaGetLastError();
}

cudaError_t launch_batch_finalize(const PageDev* pages, int n, cudaStream_t s)
{
    const int smem = static_cast<int>(sizeof(FinSmem) + sizeof(unsigned long long) * MOM_COPY_WORDS);
    cudaError_t e = cudaFuncSetAttribute(kb_fit_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kb_fit_finalize<<<static_cast<unsigned>(n), TPB, smem, s>>>(pages);
    return cudaGetLastError();
}

cudaError_t launch_pca_finalize(DevModel* dm, int B, int nvec, cudaStream_t s)
{
    const int smem = static_cast<int>(sizeof(PcaSmem));
    cudaError_t e = cudaFuncSetAttribute(k_pca_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_pca_finalize<<<1, TPB, smem, s>>>(dm, B, nvec);
    return cudaGetLastError();
}

cudaError_t launch_scatter_sb(DevModel* dm, int B, int K, cudaStream_t s)
{
    k_scatter_sb<<<1, 256, 0, s>>>(dm, B, K);
    return cudaGetLastError();
}

}  // namespace cva
