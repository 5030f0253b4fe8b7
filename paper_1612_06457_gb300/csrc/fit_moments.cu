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
// One kernel does the whole pass over the label map:
//   * each CTA walks 4096-pixel tiles (grid-stride), every thread loading 16
//     labels with one 128-bit load; tiles without a label are skipped;
//   * the tile's training pixels are bucketed by class in shared memory
//     (warp-aggregated counting sort);
//   * their band values are gathered into a shared-memory matrix of
//     augmented vectors (x_0 .. x_{B-1}, 1, 0 ..), padded to a multiple of 4;
//   * each thread owns one 4x4 block of the upper triangle of x' x'^T and a
//     stride over the pixels of one class, accumulating 16 exact products per
//     pixel (the "1" column yields n_c and s_c in the same loop);
//   * per-class block sums go to shared memory, and once per CTA to the
//     model's global moment block with 64-bit integer atomics.
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int TILE = TPB * 16;  // pixels per tile
constexpr int CHUNK = 512;      // training pixels staged per product pass

struct MomSmem {
    // dynamic part follows: acc[K][nblk][16] u64, X[CHUNK][BP] u16, sorted[TILE] u16
    int hist[MAXK];
    int start[MAXK + 1];
    int cursor[MAXK];
    unsigned char bi[MAXBLK];
    unsigned char bj[MAXBLK];
    int bad;
};

__device__ inline uint32_t label_byte(const uint4& v, int i)
{
    uint32_t w = (i < 4) ? v.x : (i < 8) ? v.y : (i < 12) ? v.z : v.w;
    return (w >> (8 * (i & 3))) & 0xFFu;
}

__global__ void __launch_bounds__(TPB)
k_fit_moments(const uint16_t* __restrict__ cube, int B, long long P,
              const uint8_t* __restrict__ labels, int K, int vec_labels,
              DevModel* __restrict__ dm)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ MomSmem sm;

    const MomShape sh = mom_shape(B);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int nacc = K * sh.nblk * 16;
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(dyn);
    uint16_t* X = reinterpret_cast<uint16_t*>(acc + nacc);
    uint16_t* sorted = X + CHUNK * sh.BP;

    for (int i = tid; i < nacc; i += TPB) acc[i] = 0ull;
    if (tid < sh.nblk) {
        // invert blk_index: walk the upper triangle in row-major order
        int idx = tid, bi = 0;
        while (idx >= sh.nb - bi) { idx -= sh.nb - bi; ++bi; }
        sm.bi[tid] = static_cast<unsigned char>(bi);
        sm.bj[tid] = static_cast<unsigned char>(bi + idx);
    }
    if (tid == 0) sm.bad = 0;

    // product-phase role of this thread: one block pair, one pixel stride
    const int G = TPB / sh.nblk;
    const int my_blk = tid % sh.nblk;
    const int my_grp = tid / sh.nblk;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    int bad = 0;

    for (long long tile = blockIdx.x; tile * TILE < P; tile += gridDim.x) {
        const long long base = tile * TILE;
        const long long p0 = base + 16LL * tid;
        uint4 lv = make_uint4(0u, 0u, 0u, 0u);
        if (vec_labels && p0 + 16 <= P) {
            lv = __ldcs(reinterpret_cast<const uint4*>(labels + p0));
        } else {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            for (int i = 0; i < 16; ++i)
                if (p0 + i < P) w[i >> 2] |= static_cast<uint32_t>(labels[p0 + i]) << (8 * (i & 3));
            lv = make_uint4(w[0], w[1], w[2], w[3]);
        }
        // labels above K are an error and are otherwise ignored
        uint32_t any = 0;
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint32_t l = label_byte(lv, i);
            if (l > static_cast<uint32_t>(K)) bad = 1;
            any |= (l != 0u && l <= static_cast<uint32_t>(K)) ? 1u : 0u;
        }
        if (tid < MAXK) sm.hist[tid] = 0;
        if (!__syncthreads_or(static_cast<int>(any))) continue;

        // --- counting sort of the tile's training pixels by class ----------
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint32_t l = label_byte(lv, i);
            if (l > static_cast<uint32_t>(K)) l = 0;
            unsigned grp = __match_any_sync(0xFFFFFFFFu, l);
            if (l != 0u && lane == __ffs(grp) - 1) atomicAdd(&sm.hist[l - 1], __popc(grp));
        }
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int c = 0; c < K; ++c) {
                sm.start[c] = run;
                sm.cursor[c] = run;
                run += sm.hist[c];
            }
            sm.start[K] = run;
        }
        __syncthreads();
        #pragma unroll
        for (int i = 0; i < 16; ++i) {
            uint32_t l = label_byte(lv, i);
            if (l > static_cast<uint32_t>(K)) l = 0;
            unsigned grp = __match_any_sync(0xFFFFFFFFu, l);
            int leader = __ffs(grp) - 1;
            int pos = 0;
            if (l != 0u && lane == leader) pos = atomicAdd(&sm.cursor[l - 1], __popc(grp));
            pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
            if (l != 0u) sorted[pos + __popc(grp & lanemask_lt)] = static_cast<uint16_t>(16 * tid + i);
        }
        __syncthreads();
        const int ntr = sm.start[K];

        // --- stage augmented vectors, then accumulate exact products -------
        for (int cs = 0; cs < ntr; cs += CHUNK) {
            const int rows = min(CHUNK, ntr - cs);
            for (int idx = tid; idx < rows * sh.BP; idx += TPB) {
                const int b = idx / rows;
                const int r = idx - b * rows;
                uint16_t v;
                if (b < B) v = __ldg(cube + static_cast<long long>(b) * P + base + sorted[cs + r]);
                else v = (b == B) ? uint16_t(1) : uint16_t(0);
                X[r * sh.BP + b] = v;
            }
            __syncthreads();
            if (my_grp < G) {
                const int bi = sm.bi[my_blk], bj = sm.bj[my_blk];
                for (int c = 0; c < K; ++c) {
                    const int s = max(sm.start[c], cs) - cs;
                    const int e = min(sm.start[c + 1], cs + rows) - cs;
                    if (s >= e) continue;
                    unsigned long long a[16];
                    #pragma unroll
                    for (int q = 0; q < 16; ++q) a[q] = 0ull;
                    for (int t = s + my_grp; t < e; t += G) {
                        const uint2 u = *reinterpret_cast<const uint2*>(X + t * sh.BP + 4 * bi);
                        const uint2 v = *reinterpret_cast<const uint2*>(X + t * sh.BP + 4 * bj);
                        const uint32_t xu[4] = {u.x & 0xFFFFu, u.x >> 16, u.y & 0xFFFFu, u.y >> 16};
                        const uint32_t xv[4] = {v.x & 0xFFFFu, v.x >> 16, v.y & 0xFFFFu, v.y >> 16};
                        #pragma unroll
                        for (int ia = 0; ia < 4; ++ia)
                            #pragma unroll
                            for (int ib = 0; ib < 4; ++ib)
                                a[4 * ia + ib] += static_cast<unsigned long long>(xu[ia] * xv[ib]);
                    }
                    unsigned long long* dst = acc + (c * sh.nblk + my_blk) * 16;
                    #pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (a[q]) atomicAdd(dst + q, a[q]);
                }
            }
            __syncthreads();
        }
    }

    if (bad) atomicOr(&sm.bad, 1);
    __syncthreads();
    for (int i = tid; i < nacc; i += TPB) {
        const unsigned long long v = acc[i];
        if (v) {
            const int c = i / (sh.nblk * 16);
            const int rest = i - c * sh.nblk * 16;
            atomicAdd(&dm->mom[c][rest / 16][rest % 16], v);
        }
    }
    if (tid == 0 && sm.bad) set_status(dm, CVA_ERR_LABEL_RANGE);
}

}  // namespace

size_t fit_moments_smem(int B, int K)
{
    const MomShape sh = mom_shape(B);
    return sizeof(unsigned long long) * K * sh.nblk * 16 + sizeof(uint16_t) * (CHUNK * sh.BP + TILE);
}

cudaError_t launch_fit_moments(const uint16_t* cube, int B, long long P, const uint8_t* labels,
                               int K, DevModel* dm, int num_sms, cudaStream_t s)
{
    const size_t smem = fit_moments_smem(B, K);
    cudaError_t e = cudaFuncSetAttribute(k_fit_moments, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fit_moments, TPB, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long tiles = (P + TILE - 1) / TILE;
    long long grid = static_cast<long long>(num_sms) * per_sm;
    if (grid > tiles) grid = tiles;
    if (grid < 1) grid = 1;
    const int vec = (reinterpret_cast<uintptr_t>(labels) % 16 == 0) ? 1 : 0;
    k_fit_moments<<<static_cast<unsigned>(grid), TPB, smem, s>>>(cube, B, P, labels, K, vec, dm);
    return cudaGetLastError();
}

}  // namespace cva
