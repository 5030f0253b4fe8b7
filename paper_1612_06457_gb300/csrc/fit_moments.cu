// fit_moments.cu -- class moments of the labelled training pixels.
//
// Section 2 of the paper builds, from the pixels the user labelled for each
// class, the within-class and between-class covariance matrices.  Both follow
// from the per-class count n_c, band sums s_c and raw second moments M_c of
// the training pixels, and because the cube holds 16-bit integers these are
// accumulated here EXACTLY in 64-bit integers: every product x_a x_b fits in
// 32 bits and the sums stay below 2^63 for H W < 2^31.  Integer sums do not
// depend on the order of accumulation, so the result is deterministic even
// though thread blocks merge their partial sums with atomics.
//
// Four kernels; the label map is cut into tiles of 16384 labels, one CTA per
// tile in the two label passes (each thread holds 64 labels from four
// 128-bit loads in flight):
//   k_tile_count    training pixels of each class in the tile, and whether
//                   the tile holds a label above K (no global atomics);
//   k_tile_scan     one CTA: prefix sums of the tile counts class by class,
//                   giving each tile its first row in every class segment of
//                   the class-major training matrix; class totals, the fit's
//                   status word, and the reset of the moment accumulators;
//   k_tile_gather   re-reads the tile, places every training pixel in its
//                   class segment (block-wide scan of packed per-thread class
//                   counts), and gathers its bands, one pixel per thread with
//                   all band loads in flight, into the augmented row
//                   (x_0 .. x_{B-1}, 1, 0 ..) of the training matrix;
//   k_moments       walks the training matrix in units of up to 256 rows of
//                   one class, staged in shared memory with 16-byte loads,
//                   and accumulates exact products, each thread owning one
//                   4x4 block of the upper triangle of x' x'^T and a stride
//                   of the unit's rows.  Sums stay in registers while a CTA
//                   stays on one class and are merged (shared memory, then
//                   global 64-bit atomics) when it moves on.  The "1" column
//                   yields n_c and s_c in the same loop.
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int TILE = LABEL_TILE;   // 16384 = TPB * 64
constexpr int SUB = TPB * 16;      // 4096 labels: one 128-bit load per thread
constexpr int UNIT = 256;          // rows per work unit of the moments pass
constexpr int NW = TPB / 32;
constexpr int LIST = 4096;         // staged training pixels per gather round
constexpr int SCAN_TPB = 1024;

// The tile's 64 labels of this thread: four 16-byte groups, SUB apart.
__device__ inline void load_tile(const uint8_t* __restrict__ labels, long long t0, long long P, int vec,
                                 uint32_t (&w)[4][4])
{
    const int tid = threadIdx.x;
    if (vec && t0 + TILE <= P) {
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(labels + t0 + u * SUB + 16LL * tid));
            w[u][0] = v.x; w[u][1] = v.y; w[u][2] = v.z; w[u][3] = v.w;
        }
    } else {
        #pragma unroll
        for (int u = 0; u < 4; ++u) {
            w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
            const long long p0 = t0 + u * SUB + 16LL * tid;
            for (int i = 0; i < 16; ++i)
                if (p0 + i < P) w[u][i >> 2] |= static_cast<uint32_t>(labels[p0 + i]) << (8 * (i & 3));
        }
    }
}

// Byte i of 16 labels held as two 64-bit halves.
__device__ inline uint32_t byte_at(unsigned long long lo, unsigned long long hi, int i)
{
    return static_cast<uint32_t>(((i < 8 ? lo : hi) >> (8 * (i & 7))) & 0xFFull);
}

// Bit i set when label byte i is a training label (1..K); `bad` when a label exceeds K.
__device__ inline uint32_t train_mask(unsigned long long lo, unsigned long long hi, int K, int& bad)
{
    uint32_t m = 0;
    #pragma unroll
    for (int i = 0; i < 16; ++i) {
        const uint32_t l = byte_at(lo, hi, i);
        m |= (l != 0u && l <= static_cast<uint32_t>(K)) ? (1u << i) : 0u;
        bad |= (l > static_cast<uint32_t>(K)) ? 1 : 0;
    }
    return m;
}

// Class counters packed four to a 64-bit word (16-bit fields; a tile holds
// 16384 labels, so no field carries into the next).
__device__ inline unsigned int field(const unsigned long long (&v)[4], int c)
{
    const unsigned long long w = (c < 4) ? v[0] : (c < 8) ? v[1] : (c < 12) ? v[2] : v[3];
    return static_cast<unsigned int>((w >> (16 * (c & 3))) & 0xFFFFull);
}

__device__ inline void bump(unsigned long long (&v)[4], int c)
{
    const unsigned long long one = 1ull << (16 * (c & 3));
    if (c < 4) v[0] += one;
    else if (c < 8) v[1] += one;
    else if (c < 12) v[2] += one;
    else v[3] += one;
}

__device__ inline unsigned int field_sum(const unsigned long long (&v)[4], int K)
{
    unsigned int s = 0;
    #pragma unroll
    for (int c = 0; c < MAXK; ++c)
        if (c < K) s += field(v, c);
    return s;
}

// Block-wide exclusive scan of packed counters (`nwords` words used).
// `wsum` is NW x 4 words of shared memory; the caller syncs before reusing it.
__device__ inline void block_scan_packed(const unsigned long long (&cnt)[4], int nwords,
                                         unsigned long long (*wsum)[4], unsigned long long (&excl)[4],
                                         unsigned long long (&total)[4])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long inc[4];
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        inc[q] = cnt[q];
        if (q < nwords) {
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, inc[q], o);
                if (lane >= o) inc[q] += v;
            }
        }
    }
    if (lane == 31) {
        #pragma unroll
        for (int q = 0; q < 4; ++q) wsum[warp][q] = inc[q];
    }
    __syncthreads();
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned long long before = 0ull, all = 0ull;
        if (q < nwords) {
            #pragma unroll
            for (int w2 = 0; w2 < NW; ++w2) {
                const unsigned long long v = wsum[w2][q];
                before += (w2 < warp) ? v : 0ull;
                all += v;
            }
        }
        excl[q] = before + inc[q] - cnt[q];
        total[q] = all;
    }
}

__global__ void __launch_bounds__(TPB)
k_tile_count(const uint8_t* __restrict__ labels, long long P, int K, int vec, unsigned int* __restrict__ tiles)
{
    __shared__ unsigned long long wsum[NW][4];
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) bad = 0;
    uint32_t w[4][4];
    load_tile(labels, static_cast<long long>(blockIdx.x) * TILE, P, vec, w);
    unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};
    int my_bad = 0;
    #pragma unroll
    for (int u = 0; u < 4; ++u) {
        const unsigned long long l64 = w[u][0] | (static_cast<unsigned long long>(w[u][1]) << 32);
        const unsigned long long h64 = w[u][2] | (static_cast<unsigned long long>(w[u][3]) << 32);
        if ((l64 | h64) == 0ull) continue;
        for (uint32_t m = train_mask(l64, h64, K, my_bad); m; m &= m - 1)
            bump(cnt, static_cast<int>(byte_at(l64, h64, __ffs(m) - 1)) - 1);
    }
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) cnt[q] += __shfl_xor_sync(0xFFFFFFFFu, cnt[q], o);
    if (lane == 0) {
        #pragma unroll
        for (int q = 0; q < 4; ++q) wsum[warp][q] = cnt[q];
    }
    __syncthreads();  // also orders the bad-flag reset before the writes below
    if (my_bad) bad = 1;
    __syncthreads();
    if (tid <= K) {
        unsigned int v;
        if (tid == K) {
            v = static_cast<unsigned int>(bad);
        } else {
            unsigned long long t[4] = {0ull, 0ull, 0ull, 0ull};
            #pragma unroll
            for (int q = 0; q < 4; ++q)
                #pragma unroll
                for (int w2 = 0; w2 < NW; ++w2) t[q] += wsum[w2][q];
            v = field(t, tid);
        }
        tiles[static_cast<long long>(blockIdx.x) * (K + 1) + tid] = v;
    }
}

__global__ void __launch_bounds__(SCAN_TPB)
k_tile_scan(int ntiles, int K, int B, long long cap, unsigned int* __restrict__ tiles, DevModel* __restrict__ dm)
{
    constexpr int SW = SCAN_TPB / 32;
    __shared__ unsigned int woff[SW][MAXK];
    __shared__ unsigned int start[MAXK];
    __shared__ int sbad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (ntiles + SCAN_TPB - 1) / SCAN_TPB;
    const int t_lo = min(ntiles, tid * per), t_hi = min(ntiles, t_lo + per);
    if (tid == 0) sbad = 0;
    unsigned int acc[MAXK];
    #pragma unroll
    for (int c = 0; c < MAXK; ++c) acc[c] = 0u;
    int bad = 0;
    for (int t = t_lo; t < t_hi; ++t) {
        const unsigned int* row = tiles + static_cast<long long>(t) * (K + 1);
        #pragma unroll
        for (int c = 0; c < MAXK; ++c)
            if (c < K) acc[c] += row[c];
        bad |= row[K] != 0u;
    }
    // exclusive scan over threads, class by class
    unsigned int ex[MAXK];
    #pragma unroll
    for (int c = 0; c < MAXK; ++c) {
        if (c < K) {
            unsigned int v = acc[c];
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int u = __shfl_up_sync(0xFFFFFFFFu, v, o);
                if (lane >= o) v += u;
            }
            ex[c] = v - acc[c];
            if (lane == 31) woff[warp][c] = v;
        } else {
            ex[c] = 0u;
        }
    }
    __syncthreads();  // also orders the bad-flag reset before the update below
    if (bad) sbad = 1;
    if (tid < K) {
        unsigned int run = 0;
        for (int w2 = 0; w2 < SW; ++w2) {
            const unsigned int v = woff[w2][tid];
            woff[w2][tid] = run;
            run += v;
        }
        dm->cls_count[tid] = run;
        start[tid] = run;  // class total for now
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long tot = 0;
        for (int c = 0; c < K; ++c) {
            const unsigned int n = start[c];
            start[c] = static_cast<unsigned int>(tot);
            tot += n;
        }
        int st = CVA_OK;
        if (sbad) st = CVA_ERR_LABEL_RANGE;
        else if (tot > static_cast<unsigned long long>(cap)) st = CVA_ERR_CAPACITY;
        dm->status = st;
        dm->fitted = 0;
    }
    __syncthreads();
    // each tile's first row in every class segment (in place of its counts)
    unsigned int run[MAXK];
    #pragma unroll
    for (int c = 0; c < MAXK; ++c) run[c] = (c < K) ? start[c] + woff[warp][c] + ex[c] : 0u;
    for (int t = t_lo; t < t_hi; ++t) {
        unsigned int* row = tiles + static_cast<long long>(t) * (K + 1);
        #pragma unroll
        for (int c = 0; c < MAXK; ++c) {
            if (c < K) {
                const unsigned int n = row[c];
                row[c] = run[c];
                run[c] += n;
            }
        }
    }
    // reset the moment accumulators of this fit
    const MomShape sh = mom_shape(B);
    for (int i = tid; i < K * sh.nblk * 16; i += SCAN_TPB) {
        const int c = i / (sh.nblk * 16), rest = i - c * sh.nblk * 16;
        dm->mom[c][rest >> 4][rest & 15] = 0ull;
    }
}

__global__ void __launch_bounds__(TPB)
k_tile_gather(const uint16_t* __restrict__ cube, int B, long long P, const uint8_t* __restrict__ labels, int K,
              int vec, const unsigned int* __restrict__ tiles, uint16_t* __restrict__ xtr,
              const DevModel* __restrict__ dm)
{
    __shared__ unsigned long long wsum[NW][4];
    __shared__ unsigned int base[MAXK];
    __shared__ unsigned int lp[LIST], lr[LIST];
    __shared__ int nlist;
    const int tid = threadIdx.x;
    if (dm->status != 0) return;
    const long long t0 = static_cast<long long>(blockIdx.x) * TILE;
    uint32_t w[4][4];
    load_tile(labels, t0, P, vec, w);
    if (tid < K) base[tid] = tiles[static_cast<long long>(blockIdx.x) * (K + 1) + tid];
    if (tid == 0) nlist = 0;
    const int nwords = (K + 3) >> 2;
    const int BR = xtr_row(B);

    auto gather = [&](int n) {
        for (int i = tid; i < n; i += TPB) {
            const uint16_t* src = cube + lp[i];
            uint32_t xv[MAXB];
            #pragma unroll
            for (int b = 0; b < MAXB; ++b) xv[b] = (b < B) ? static_cast<uint32_t>(__ldg(src + static_cast<long long>(b) * P)) : 0u;
            uint4* grow = reinterpret_cast<uint4*>(xtr + static_cast<long long>(lr[i]) * BR);
            #pragma unroll
            for (int q = 0; q < (MAXB + 8) / 8; ++q) {
                if (q * 8 < BR) {
                    uint32_t pk[4];
                    #pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int b0 = q * 8 + 2 * h, b1 = b0 + 1;
                        const uint32_t v0 = (b0 < B) ? xv[b0 < MAXB ? b0 : 0] : (b0 == B ? 1u : 0u);
                        const uint32_t v1 = (b1 < B) ? xv[b1 < MAXB ? b1 : 0] : (b1 == B ? 1u : 0u);
                        pk[h] = v0 | (v1 << 16);
                    }
                    grow[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
        }
    };

    int bad_unused = 0;
    #pragma unroll
    for (int u = 0; u < 4; ++u) {
        const unsigned long long l64 = w[u][0] | (static_cast<unsigned long long>(w[u][1]) << 32);
        const unsigned long long h64 = w[u][2] | (static_cast<unsigned long long>(w[u][3]) << 32);
        const uint32_t mask = (l64 | h64) ? train_mask(l64, h64, K, bad_unused) : 0u;
        if (!__syncthreads_or(mask != 0u)) continue;
        unsigned long long cnt[4] = {0ull, 0ull, 0ull, 0ull};
        for (uint32_t m = mask; m; m &= m - 1) bump(cnt, static_cast<int>(byte_at(l64, h64, __ffs(m) - 1)) - 1);
        unsigned long long excl[4], total[4];
        block_scan_packed(cnt, nwords, wsum, excl, total);
        const unsigned int sub_n = field_sum(total, K);
        if (nlist + static_cast<int>(sub_n) > LIST) {  // uniform: make room first
            gather(nlist);
            __syncthreads();
            if (tid == 0) nlist = 0;
            __syncthreads();
        }
        // slot in the staging list: pixels of this thread after those of lower threads
        unsigned int slot = static_cast<unsigned int>(nlist) + field_sum(excl, K);
        unsigned long long run[4] = {excl[0], excl[1], excl[2], excl[3]};
        const long long p0 = t0 + u * SUB + 16LL * tid;
        for (uint32_t m = mask; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            const int c = static_cast<int>(byte_at(l64, h64, i)) - 1;
            lp[slot] = static_cast<unsigned int>(p0 + i);
            lr[slot] = base[c] + field(run, c);
            bump(run, c);
            ++slot;
        }
        __syncthreads();
        if (tid < K) base[tid] += field(total, tid);
        if (tid == 0) nlist += static_cast<int>(sub_n);
        __syncthreads();
    }
    gather(nlist);
}

__global__ void __launch_bounds__(TPB)
k_moments(int B, int K, const uint16_t* __restrict__ xtr, long long cap, DevModel* __restrict__ dm)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned int ustart[MAXK + 1], cstart[MAXK], ccount[MAXK];
    __shared__ unsigned char sbi[MAXBLK], sbj[MAXBLK];
    __shared__ int stop;

    const MomShape sh = mom_shape(B);
    const int BR = xtr_row(B);
    const int tid = threadIdx.x;
    const int G = TPB / sh.nblk;
    uint16_t* X = reinterpret_cast<uint16_t*>(dyn);                                            // UNIT x BR
    unsigned long long* part = reinterpret_cast<unsigned long long*>(dyn + UNIT * BR * 2);     // G x nblk x 16

    if (tid == 0) {
        unsigned int run = 0, units = 0;
        unsigned long long tot = 0;
        for (int c = 0; c < K; ++c) {
            const unsigned int n = dm->cls_count[c];
            cstart[c] = run;
            ccount[c] = n;
            ustart[c] = units;
            run += n;
            tot += n;
            units += (n + UNIT - 1) / UNIT;
        }
        ustart[K] = units;
        stop = (dm->status != 0) || (tot > static_cast<unsigned long long>(cap));
    }
    if (tid < sh.nblk) {
        int idx = tid, bi = 0;
        while (idx >= sh.nb - bi) { idx -= sh.nb - bi; ++bi; }
        sbi[tid] = static_cast<unsigned char>(bi);
        sbj[tid] = static_cast<unsigned char>(bi + idx);
    }
    __syncthreads();
    if (stop) return;

    const int my_blk = tid % sh.nblk;
    const int my_grp = tid / sh.nblk;
    const bool worker = my_grp < G;
    const int bi = worker ? sbi[my_blk] : 0, bj = worker ? sbj[my_blk] : 0;
    unsigned long long a[16];
    #pragma unroll
    for (int q = 0; q < 16; ++q) a[q] = 0ull;
    int cur_class = -1;

    auto flush = [&](int c) {
        if (worker) {
            unsigned long long* dst = part + (my_grp * sh.nblk + my_blk) * 16;
            #pragma unroll
            for (int q = 0; q < 16; ++q) { dst[q] = a[q]; a[q] = 0ull; }
        }
        __syncthreads();
        for (int i = tid; i < sh.nblk * 16; i += TPB) {
            unsigned long long v = 0ull;
            for (int g = 0; g < G; ++g) v += part[g * sh.nblk * 16 + i];
            if (v) atomicAdd(&dm->mom[c][i >> 4][i & 15], v);
        }
        __syncthreads();
    };

    const unsigned int nunits = ustart[K];
    const int vec_per_row = BR / 8;
    for (unsigned int u = blockIdx.x; u < nunits; u += gridDim.x) {
        int c = 0;
        while (u >= ustart[c + 1]) ++c;
        if (c != cur_class) {
            if (cur_class >= 0) flush(cur_class);
            cur_class = c;
        }
        const unsigned int row0 = cstart[c] + (u - ustart[c]) * UNIT;
        const int len = static_cast<int>(min(static_cast<unsigned int>(UNIT), cstart[c] + ccount[c] - row0));
        const uint4* src = reinterpret_cast<const uint4*>(xtr + static_cast<long long>(row0) * BR);
        uint4* dst = reinterpret_cast<uint4*>(X);
        for (int i = tid; i < len * vec_per_row; i += TPB) dst[i] = __ldg(src + i);
        __syncthreads();
        if (worker) {
            for (int t = my_grp; t < len; t += G) {
                const uint2 uu = *reinterpret_cast<const uint2*>(X + t * BR + 4 * bi);
                const uint2 vv = *reinterpret_cast<const uint2*>(X + t * BR + 4 * bj);
                const uint32_t xu[4] = {uu.x & 0xFFFFu, uu.x >> 16, uu.y & 0xFFFFu, uu.y >> 16};
                const uint32_t xw[4] = {vv.x & 0xFFFFu, vv.x >> 16, vv.y & 0xFFFFu, vv.y >> 16};
                #pragma unroll
                for (int ia = 0; ia < 4; ++ia)
                    #pragma unroll
                    for (int ib = 0; ib < 4; ++ib)
                        a[4 * ia + ib] += static_cast<unsigned long long>(xu[ia]) * xw[ib];
            }
        }
        __syncthreads();
    }
    if (cur_class >= 0) flush(cur_class);
}

}  // namespace

cudaError_t launch_fit_moments(const uint16_t* cube, int B, long long P, const uint8_t* labels, int K,
                               DevModel* dm, uint16_t* xtr, unsigned int* tiles, long long cap, int num_sms,
                               cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(labels) % 16 == 0) ? 1 : 0;
    const long long ntiles = (P + TILE - 1) / TILE;
    k_tile_count<<<static_cast<unsigned>(ntiles), TPB, 0, s>>>(labels, P, K, vec, tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_scan<<<1, SCAN_TPB, 0, s>>>(static_cast<int>(ntiles), K, B, cap, tiles, dm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tile_gather<<<static_cast<unsigned>(ntiles), TPB, 0, s>>>(cube, B, P, labels, K, vec, tiles, xtr, dm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    const MomShape sh = mom_shape(B);
    const int G = TPB / sh.nblk;
    const size_t smem = static_cast<size_t>(UNIT) * xtr_row(B) * 2 + static_cast<size_t>(G) * sh.nblk * 16 * 8;
    e = cudaFuncSetAttribute(k_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    // the unit count is only known on the device: size the grid for the
    // useful maximum and let idle CTAs exit at once
    const long long g3 = static_cast<long long>(num_sms) * 4;
    k_moments<<<static_cast<unsigned>(g3), TPB, smem, s>>>(B, K, xtr, cap, dm);
    return cudaGetLastError();
}

}  // namespace cva
