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
// Two passes for one page after a one-CTA reset (k_fit_reset):
//   k_label_scan      one pass over the labels: each warp takes 512 labels at
//                     a time (one 16-byte load a lane) and, converged, stages
//                     the labelled ones in shared memory by ballots, counts
//                     them by class with one ballot per class, reserves their
//                     rows with one atomic per class (lane c for class c) and
//                     writes every pixel index to its class's region of the
//                     list (class c at list + c cap, in no fixed order);
//   k_gather_moments  one CTA per unit of up to 256 training rows of one
//                     class: the rows' bands gathered from the cube (one pixel
//                     a thread, all band loads in flight), written to the
//                     class-major training matrix (16-byte rows
//                     (x_0 .. x_{B-1}, 1, 0 ..), read by the training-range
//                     pass) and, split into bytes, to shared memory, then the
//                     exact moments on the tensor cores (see the kernel).
//                     Sums stay in registers while a CTA stays on one class
//                     and are merged into the model with 64-bit integer
//                     atomics when it moves on.  The "1" column yields n_c
//                     and s_c in the same pass.
// Training pixels are a small share of a page, so loops of each lane over its
// own labels would leave most lanes idle: the label passes stay converged on
// the warp and their cost is the labels' one read plus a little work per
// chunk that holds a training pixel.
// The same passes in batched form (kb_*: the flattened work of many pages,
// see batch.cu), where the training lists are sized exactly: a count pass
// over tiles of 16384 labels (the same staged chunks; each page's last CTA
// takes the prefix sums over its tiles) and a compaction pass that reserves
// each chunk's rows inside its tile's share with shared-memory atomics; and
// the moments of every selected pixel of a page for the
// principal components (k_pca_moments, straight from the cube).
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int TILE = LABEL_TILE;   // 16384 = TPB * 64
constexpr int SUB = TPB * 16;      // 4096 labels: one 128-bit load per thread
constexpr int NG = TILE / SUB;     // 16-label groups (128-bit loads) per thread: 4
constexpr int UNIT = 256;          // rows per work unit of the moments pass
constexpr int NW = TPB / 32;

// The tile's 64 labels of this thread: NG 16-byte groups, SUB apart.
__device__ inline void load_tile(const uint8_t* __restrict__ labels, long long t0, long long P, int vec,
                                 uint32_t (&w)[NG][4])
{
    const int tid = threadIdx.x;
    if (vec && t0 + TILE <= P) {
        #pragma unroll
        for (int u = 0; u < NG; ++u) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(labels + t0 + u * SUB + 16LL * tid));
            w[u][0] = v.x; w[u][1] = v.y; w[u][2] = v.z; w[u][3] = v.w;
        }
    } else {
        #pragma unroll
        for (int u = 0; u < NG; ++u) {
            w[u][0] = w[u][1] = w[u][2] = w[u][3] = 0u;
            const long long p0 = t0 + u * SUB + 16LL * tid;
            for (int i = 0; i < 16; ++i)
                if (p0 + i < P) w[u][i >> 2] |= static_cast<uint32_t>(labels[p0 + i]) << (8 * (i & 3));
        }
    }
}

// Prefix sums of the per-tile class counts (run by one CTA): each tile's
// count of class c becomes its first row within the class c segment of the
// class-major training list (the segment's own start is added by the
// compaction pass).  The tile rows are staged through shared memory in
// chunks, one coalesced load and store per chunk, and scanned there with one
// warp per class.  Also the label check, the class totals, the fit's status
// word and the reset of the moment accumulators.
constexpr int SCAN_CHUNK = 4096;  // words of tile rows per chunk

__device__ void scan_tiles(int ntiles, int K, int B, long long cap, unsigned int* __restrict__ tiles,
                           DevModel* __restrict__ dm)
{
    __shared__ unsigned int buf[SCAN_CHUNK];
    __shared__ unsigned int carry[MAXK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row = K + 1;
    const int per_chunk = SCAN_CHUNK / row;
    if (tid < K) carry[tid] = 0u;
    int bad = 0;
    for (int t0 = 0; t0 < ntiles; t0 += per_chunk) {
        const int nt = min(per_chunk, ntiles - t0);
        const int nw = nt * row;
        const long long g0 = static_cast<long long>(t0) * row;
        __syncthreads();  // carry set; the previous chunk's buf written out
        for (int i = tid; i < nw; i += TPB) buf[i] = __ldcg(tiles + g0 + i);
        __syncthreads();
        for (int t = tid; t < nt; t += TPB) bad |= buf[t * row + K] != 0u;
        const int per = (nt + 31) / 32;
        const int a = min(nt, lane * per), e = min(nt, a + per);
        for (int c = warp; c < K; c += NW) {
            unsigned int acc = 0;
            for (int t = a; t < e; ++t) acc += buf[t * row + c];
            unsigned int v = acc;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned int u = __shfl_up_sync(0xFFFFFFFFu, v, o);
                if (lane >= o) v += u;
            }
            unsigned int run = carry[c] + v - acc;
            for (int t = a; t < e; ++t) {
                const unsigned int n = buf[t * row + c];
                buf[t * row + c] = run;
                run += n;
            }
            __syncwarp();
            if (lane == 31) carry[c] += v;
        }
        __syncthreads();
        for (int i = tid; i < nw; i += TPB) tiles[g0 + i] = buf[i];
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        unsigned long long total = 0;
        for (int c = 0; c < K; ++c) {
            dm->cls_count[c] = carry[c];
            total += carry[c];
        }
        int st = CVA_OK;
        if (bad) st = CVA_ERR_LABEL_RANGE;
        else if (total > static_cast<unsigned long long>(cap)) st = CVA_ERR_CAPACITY;
        dm->status = st;
        dm->fitted = 0;
        dm->tile_ticket = 0u;
    }
    const MomShape sh = mom_shape(B);
    for (int i = tid; i < K * sh.nblk * 16; i += TPB) {
        const int c = i / (sh.nblk * 16), rest = i - c * sh.nblk * 16;
        dm->mom[c][rest >> 4][rest & 15] = 0ull;
    }
}

// The labelled pixels of one warp's 512 labels (16 a lane, in w) staged in
// `st` in (byte position, lane) order, one ballot per byte position; an
// entry is the pixel's offset in the 512 | its label << 16.  Returns how many.
// Every lane of the warp calls it; st is read after it returns.
__device__ __forceinline__ int stage_chunk(const uint32_t (&w)[4], uint32_t* st, int lane)
{
    const uint32_t below = (1u << lane) - 1u;
    int T = 0;
    #pragma unroll
    for (int j = 0; j < 16; ++j) {
        const uint32_t v = (w[j >> 2] >> (8 * (j & 3))) & 0xFFu;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, v != 0u);
        if (bal) {
            if (v) st[T + __popc(bal & below)] = static_cast<uint32_t>(16 * lane + j) | (v << 16);
            T += __popc(bal);
        }
    }
    __syncwarp();
    return T;
}

// Class counts of T staged entries, one ballot per class and 32 entries:
// added to `mine` on lane c for class c.  Sets `over` for a label above K.
__device__ __forceinline__ void count_staged(const uint32_t* st, int T, int K, int lane, unsigned int& mine, bool& over)
{
    for (int i0 = 0; i0 < T; i0 += 32) {
        const uint32_t v = (i0 + lane < T) ? (st[i0 + lane] >> 16) : 0u;
        over |= v > static_cast<uint32_t>(K);
        for (int c = 0; c < K; ++c) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, v == static_cast<uint32_t>(c + 1));
            if (lane == c) mine += __popc(bal);
        }
    }
}

// Rows for T staged entries: class c's next row is lane c's `run` (advanced
// past them); each entry goes to list[c * stride + row] as p0 + its offset.
__device__ __forceinline__ void place_staged(const uint32_t* st, int T, int K, int lane, unsigned int run,
                                             unsigned long long p0, unsigned int* __restrict__ list,
                                             long long stride, long long cap)
{
    const uint32_t below = (1u << lane) - 1u;
    for (int i0 = 0; i0 < T; i0 += 32) {
        const uint32_t e = (i0 + lane < T) ? st[i0 + lane] : 0u;
        const uint32_t v = e >> 16;
        for (int c = 0; c < K; ++c) {
            const uint32_t bal = __ballot_sync(0xFFFFFFFFu, v == static_cast<uint32_t>(c + 1));
            const unsigned int base = __shfl_sync(0xFFFFFFFFu, run, c);
            if (v == static_cast<uint32_t>(c + 1)) {
                const unsigned long long pos = static_cast<unsigned long long>(base) + __popc(bal & below);
                if (pos < static_cast<unsigned long long>(cap))
                    list[static_cast<long long>(c) * stride + static_cast<long long>(pos)] =
                        static_cast<unsigned int>(p0 + (e & 0xFFFFu));
            }
            if (lane == c) run += __popc(bal);
        }
    }
}

// One tile's class counts (tile `tile` of the page); the page's last CTA to
// finish takes the prefix sums.
__device__ __forceinline__ void tile_count_body(const uint8_t* __restrict__ labels, long long P, int K, int B, int vec,
                                                long long cap, int ntiles, unsigned int* __restrict__ tiles,
                                                DevModel* __restrict__ dm, int tile)
{
    __shared__ uint32_t stage[NW][512];
    __shared__ unsigned int scnt[MAXK];
    __shared__ int bad;
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < MAXK) scnt[tid] = 0u;
    if (tid == 0) bad = 0;
    uint32_t w[NG][4];
    load_tile(labels, static_cast<long long>(tile) * TILE, P, vec, w);
    __syncthreads();
    // warp w's chunks: labels u SUB + 512 w .. + 511 of the tile, u < NG
    unsigned int mine = 0u;
    bool over = false;
    #pragma unroll
    for (int u = 0; u < NG; ++u) {
        if (!__any_sync(0xFFFFFFFFu, (w[u][0] | w[u][1] | w[u][2] | w[u][3]) != 0u)) continue;
        const int T = stage_chunk(w[u], stage[warp], lane);
        count_staged(stage[warp], T, K, lane, mine, over);
        __syncwarp();  // the stage is rewritten by the next chunk
    }
    if (lane < K && mine) atomicAdd(&scnt[lane], mine);
    if (__any_sync(0xFFFFFFFFu, over) && lane == 0) bad = 1;
    __syncthreads();
    if (tid <= K) tiles[static_cast<long long>(tile) * (K + 1) + tid] = (tid == K) ? static_cast<unsigned int>(bad) : scnt[tid];
    // the last CTA to finish (atomic ticket after a fence) scans the counts;
    // no CTA ever waits for another
    __threadfence();
    __syncthreads();
    if (tid == 0) last = (atomicAdd(&dm->tile_ticket, 1u) == static_cast<unsigned int>(ntiles - 1));
    __syncthreads();
    if (!last) return;
    __threadfence();
    scan_tiles(ntiles, K, B, cap, tiles, dm);
}

// One tile's training pixels written to their rows of the class-major list.
// `cls_count` gives the class segment starts, `tiles` each tile's first row
// within every segment.
__device__ __forceinline__ void tile_compact_body(const uint8_t* __restrict__ labels, long long P, int K, int vec,
                                                  const unsigned int* __restrict__ tiles,
                                                  const unsigned int* __restrict__ cls_count,
                                                  unsigned int* __restrict__ list, int tile)
{
    __shared__ uint32_t stage[NW][512];
    __shared__ unsigned int base[MAXK];  // next free row of each class in this tile's share
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t0 = static_cast<long long>(tile) * TILE;
    uint32_t w[NG][4];
    load_tile(labels, t0, P, vec, w);
    if (tid < K) {
        unsigned int start = 0;
        for (int c = 0; c < tid; ++c) start += cls_count[c];
        base[tid] = start + tiles[static_cast<long long>(tile) * (K + 1) + tid];
    }
    __syncthreads();
    // each chunk reserves its rows of every class with one shared-memory
    // atomic (lane c for class c) and places its pixels by ballots
    #pragma unroll
    for (int u = 0; u < NG; ++u) {
        if (!__any_sync(0xFFFFFFFFu, (w[u][0] | w[u][1] | w[u][2] | w[u][3]) != 0u)) continue;
        const int T = stage_chunk(w[u], stage[warp], lane);
        unsigned int mine = 0u;
        bool over = false;
        count_staged(stage[warp], T, K, lane, mine, over);
        const unsigned int run = (lane < K && mine) ? atomicAdd(&base[lane], mine) : 0u;
        place_staged(stage[warp], T, K, lane, run, static_cast<unsigned long long>(t0 + u * SUB + 512 * warp), list,
                     0, 0x7FFFFFFFFFFFFFFFll);
        __syncwarp();  // the stage is rewritten by the next chunk
    }
}

// A read-only 16-bit load that asks L2 to fetch 64 bytes around it: the
// training pixels sit in short runs (4-23 pixels on average per class on the
// benchmark page), so the default fetches mostly bring unused bytes; measured
// on the 23-band 4096 x 4096 page the gather's DRAM reads drop from 74 MB to
// 43 MB (the distinct 64-byte blocks its values occupy: 42.4 MB; 32-byte
// sectors: 26.1 MB) at the same kernel time, which is bound by load latency.
__device__ inline uint32_t ld_u16_l2_64(const uint16_t* p)
{
    unsigned short v;
    asm volatile("ld.global.nc.L2::64B.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

// The fit's state before the label scan: moments and class counters zero,
// status clear, model not fitted (one CTA).
__global__ void k_fit_reset(DevModel* __restrict__ dm, int B, int K)
{
    const MomShape sh = mom_shape(B);
    for (int i = threadIdx.x; i < K * sh.nblk * 16; i += blockDim.x) {
        const int c = i / (sh.nblk * 16), rest = i - c * sh.nblk * 16;
        dm->mom[c][rest >> 4][rest & 15] = 0ull;
    }
    if (threadIdx.x < MAXK) dm->cls_count[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        dm->status = CVA_OK;
        dm->fitted = 0;
    }
}

// One warp's 16-byte share (lane `lane`) of the 512-label chunk `ch`; zero
// past the page's end.
__device__ __forceinline__ uint4 chunk_load(const uint8_t* __restrict__ labels, long long P, int vec, long long ch,
                                            int lane)
{
    const long long p0 = ch * 512 + 16LL * lane;
    if (vec && ch * 512 + 512 <= P) return __ldcs(reinterpret_cast<const uint4*>(labels + p0));
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    for (int i = 0; i < 16; ++i)
        if (p0 + i < P) w[i >> 2] |= static_cast<uint32_t>(labels[p0 + i]) << (8 * (i & 3));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// One pass over the labels: the index of every training pixel goes to its
// class's region of the list (class c at list + c cap, in no particular
// order).  Each warp takes 512 labels at a time (16 a lane, one 16-byte load,
// the next chunk's load in flight) and skips them when none is set.  The
// training pixels are a small part of a page, and per-lane loops over them
// leave most lanes idle, so everything runs converged on the warp:
//   * one ballot per byte position compacts the chunk's labelled pixels into
//     the warp's staging area in shared memory (pixel offset | label << 16);
//   * 32 entries at a time, one ballot per class counts them, lane c adds the
//     chunk's count of class c to that class's counter (all classes' atomics
//     in flight together), and the same ballots again give every entry its
//     row: the class's base plus its rank among the lanes below it.
// The moments are exact integer sums and the ranges minima and maxima, so
// nothing downstream depends on the order.  A label above K sets
// CVA_ERR_LABEL_RANGE and is not listed; entries beyond cap are dropped (the
// gather-moments pass then reports CVA_ERR_CAPACITY).
__global__ void __launch_bounds__(TPB)
k_label_scan(const uint8_t* __restrict__ labels, long long P, int K, int vec, long long cap,
             unsigned int* __restrict__ list, DevModel* __restrict__ dm)
{
    __shared__ uint32_t stage[NW][512];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nchunk = (P + 511) / 512;
    const long long wid = (static_cast<long long>(blockIdx.x) * TPB + threadIdx.x) >> 5;
    const long long nw = (static_cast<long long>(gridDim.x) * TPB) >> 5;
    uint32_t* st = stage[warp];
    bool bad = false;
    long long ch = wid;
    uint4 next = make_uint4(0u, 0u, 0u, 0u);
    if (ch < nchunk) next = chunk_load(labels, P, vec, ch, lane);
    for (; ch < nchunk; ch += nw) {  // the same for every lane of the warp
        const uint4 x = next;
        if (ch + nw < nchunk) next = chunk_load(labels, P, vec, ch + nw, lane);
        if (!__any_sync(0xFFFFFFFFu, (x.x | x.y | x.z | x.w) != 0u)) continue;
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
        const int T = stage_chunk(w, st, lane);
        unsigned int mine = 0u;  // lane c: the chunk's count of class c
        count_staged(st, T, K, lane, mine, bad);
        // lane c reserves class c's rows (all classes' atomics in flight together)
        const unsigned int run = (lane < K && mine) ? atomicAdd(&dm->cls_count[lane], mine) : 0u;
        place_staged(st, T, K, lane, run, static_cast<unsigned long long>(ch * 512), list, cap, cap);
        __syncwarp();  // the staging area is rewritten by the next chunk
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) atomicCAS(&dm->status, 0, CVA_ERR_LABEL_RANGE);
}

// ldmatrix / mma.sync wrappers (bf16 inputs, f32 accumulators)
__device__ inline void ldsm_x4(uint32_t (&r)[4], const void* smem)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ inline void ldsm_x2(uint32_t (&r)[2], const void* smem)
{
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

__device__ inline void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// bf16 bit pattern of an integer 0 <= v < 256 (exact: at most 8 significant bits).
__device__ inline uint32_t bf16_of_byte(uint32_t v)
{
    return __float_as_uint(static_cast<float>(v)) >> 16;
}

constexpr int UPAD = UNIT + 8;  // shared row stride (bf16) of the transposed unit: conflict-free ldmatrix
constexpr int MAXPAIR = MAXBA * (MAXBA + 1) / 2;

// (a, b) of every upper-triangle entry a <= b of the (B+1) x (B+1) augmented
// moment matrix, in row-major order.
__device__ __forceinline__ void build_pairs(unsigned char* pa, unsigned char* pb, int BA)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int a = warp; a < BA; a += NW)
        for (int b = a + lane; b < BA; b += 32) {
            const int q = a * BA - a * (a - 1) / 2 + (b - a);
            pa[q] = static_cast<unsigned char>(a);
            pb[q] = static_cast<unsigned char>(b);
        }
}

// Merge a thread's (up to three) moment sums into class c of the model.
__device__ __forceinline__ void moments_flush(DevModel* __restrict__ dm, int c, int nb, int npair,
                                              const unsigned char* pa, const unsigned char* pb,
                                              unsigned long long (&acc)[3])
{
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = threadIdx.x + k * TPB;
        if (q < npair && acc[k]) {
            const int a = pa[q], b = pb[q];
            atomicAdd(&dm->mom[c][blk_index(a >> 2, b >> 2, nb)][(a & 3) * 4 + (b & 3)], acc[k]);
        }
        acc[k] = 0ull;
    }
}

// Row stride (floats) of the Gram matrix in shared memory: odd, so that the
// strided reads below spread over the banks.
__host__ __device__ constexpr int cs_stride(int F2) { return F2 + 1; }

// Dynamic shared memory of the moment kernels for padded width F: the split
// matrix and the Gram matrix.
__host__ __device__ constexpr size_t moments_smem_bytes(int F)
{
    return static_cast<size_t>(2 * F) * UPAD * 2 + static_cast<size_t>(2 * F) * cs_stride(2 * F) * 4;
}

// The Gram matrix of a staged unit (XT: the (2 F) x 256 split matrix [h ; l]
// in shared memory) on the tensor cores, added to the thread's moment sums.
// A warp task is one 16-row block against two 8-column blocks, so each A
// fragment feeds two mma (two independent accumulator chains); the Gram
// matrix is symmetric and only entries on or above the diagonal are read, so
// tasks wholly below it are skipped.  Every thread of the CTA takes part (two
// barriers; the caller synchronizes after staging).
__device__ __forceinline__ void moments_gram(const uint16_t* XT, float* Cs, int F, int npair, const unsigned char* pa,
                                             const unsigned char* pb, unsigned long long (&acc)[3])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int F2 = 2 * F, CS = cs_stride(F2);
    const int MT = F2 / 16, NP = F2 / 16;  // 16-row blocks, pairs of 8-column blocks
    for (int t = warp; t < MT * NP; t += NW) {
        const int mt = t / NP, np = t - (t / NP) * NP;
        if (np * 16 + 15 < mt * 16) continue;
        // every partial sum is an integer below 2^24: exact in FP32
        float d0[4] = {0.0f, 0.0f, 0.0f, 0.0f}, d1[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const uint16_t* arow = XT + (mt * 16 + (lane & 15)) * UPAD + ((lane >> 4) << 3);
        const uint16_t* brow0 = XT + (np * 16 + (lane & 7)) * UPAD + (((lane >> 3) & 1) << 3);
        const uint16_t* brow1 = brow0 + 8 * UPAD;
        #pragma unroll 4
        for (int ks = 0; ks < UNIT / 16; ++ks) {
            uint32_t af[4], b0[2], b1[2];
            ldsm_x4(af, arow + ks * 16);
            ldsm_x2(b0, brow0 + ks * 16);
            ldsm_x2(b1, brow1 + ks * 16);
            mma_bf16_16816(d0, af, b0);
            mma_bf16_16816(d1, af, b1);
        }
        const int r0 = mt * 16 + (lane >> 2), c0 = np * 16 + (lane & 3) * 2;
        Cs[r0 * CS + c0] = d0[0];
        Cs[r0 * CS + c0 + 1] = d0[1];
        Cs[(r0 + 8) * CS + c0] = d0[2];
        Cs[(r0 + 8) * CS + c0 + 1] = d0[3];
        Cs[r0 * CS + c0 + 8] = d1[0];
        Cs[r0 * CS + c0 + 9] = d1[1];
        Cs[(r0 + 8) * CS + c0 + 8] = d1[2];
        Cs[(r0 + 8) * CS + c0 + 9] = d1[3];
    }
    __syncthreads();
    #pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int q = tid + k * TPB;
        if (q < npair) {
            const int a = pa[q], b = pb[q];
            const unsigned long long hh = __float2uint_rn(Cs[a * CS + b]);
            const unsigned long long hl = __float2uint_rn(Cs[a * CS + F + b]);
            const unsigned long long lh = __float2uint_rn(Cs[b * CS + F + a]);  // = C[F + a][b] by symmetry
            const unsigned long long ll = __float2uint_rn(Cs[(F + a) * CS + F + b]);
            acc[k] += (hh << 16) + ((hl + lh) << 8) + ll;
        }
    }
    __syncthreads();
}

// One unit's training pixels gathered and staged: thread t < len takes
// pixel ulist[t] of the cube (all band loads in flight, with the gather's
// 64-byte fetch hint), writes its augmented row (x_0 .. x_{B-1}, 1, zeros) to
// rows + t F and its bytes to the transposed unit XT; threads from len on
// stage zero columns.  NBAND (24 or MAXB) bounds B.  The caller
// synchronizes before XT is read.
template <int NBAND>
__device__ __forceinline__ void gather_stage(uint16_t* XT, const uint16_t* __restrict__ cube, int B, long long P,
                                             const unsigned int* __restrict__ ulist, uint16_t* __restrict__ rows,
                                             int F, int len)
{
    const int tid = threadIdx.x;
    const bool live = tid < len;
    uint32_t xv[NBAND];
    if (live) {
        const uint16_t* src = cube + ulist[tid];
        #pragma unroll
        for (int b = 0; b < NBAND; ++b) xv[b] = (b < B) ? ld_u16_l2_64(src + static_cast<long long>(b) * P) : 0u;
    } else {
        #pragma unroll
        for (int b = 0; b < NBAND; ++b) xv[b] = 0u;
    }
    uint4* grow = reinterpret_cast<uint4*>(rows + static_cast<long long>(tid) * F);
    #pragma unroll
    for (int q = 0; q < (NBAND + 8) / 8; ++q) {
        if (q * 8 < F) {
            uint32_t pk[4];
            #pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int f = q * 8 + h;
                uint32_t v = (f < B) ? xv[f < NBAND ? f : 0] : (f == B ? 1u : 0u);
                if (!live) v = 0u;
                if (h & 1) pk[h >> 1] |= v << 16;
                else pk[h >> 1] = v;
                XT[f * UPAD + tid] = static_cast<uint16_t>(bf16_of_byte(v >> 8));
                XT[(F + f) * UPAD + tid] = static_cast<uint16_t>(bf16_of_byte(v & 0xFFu));
            }
            if (live) grow[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// Exact moments on the tensor cores.  A unit holds up to 256 training rows of
// one class.  Every 16-bit value x is split into its high and low bytes,
// x = 256 h + l, both exact in bf16; the unit is stored transposed in shared
// memory as the (2 F) x 256 matrix [h ; l] (F = padded augmented width), and
// mma.sync forms its Gram matrix C = [h ; l] [h ; l]^T with FP32 accumulation.
// Every partial sum is an integer below 256 * 255^2 < 2^24, so C is exact, and
//     sum x_a x_b = 65536 C_hh[a][b] + 256 (C_hl[a][b] + C_lh[a][b]) + C_ll[a][b]
// is recombined in 64-bit integers.  Each thread owns up to three (a <= b)
// entries of the augmented moment matrix and keeps them in registers while
// the CTA stays on one class.
//
// For one page the gather is fused with the moments: one CTA per unit of up
// to 256 training rows of one class, and thread t takes the unit's pixel t
// straight from the cube (all NBAND band loads in flight, with the 64-byte
// fetch hint of the gather), writes its augmented row to the training matrix
// (which the training-range pass reads) and its bytes to the transposed unit
// in shared memory, from which the Gram matrix is formed.  Against a gather
// pass and a moments pass (18 + 12.4 us under ncu on the benchmark page) it
// takes 23.5-24.8 us: one launch and the training matrix's re-read fewer.  NBAND
// (24 or MAXB) bounds B, so that the 23-band case keeps 24 values a thread:
// 48 registers, five CTAs an SM (with six the values spill); four above 24.
__host__ __device__ constexpr int gm_ctas(int NBAND) { return NBAND <= 24 ? 5 : 4; }

template <int NBAND>
__global__ void __launch_bounds__(TPB, gm_ctas(NBAND))
k_gather_moments(const uint16_t* __restrict__ cube, int B, long long P, int K, const unsigned int* __restrict__ list,
                 long long cap, uint16_t* __restrict__ xtr, DevModel* __restrict__ dm)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned int ustart[MAXK + 1], cstart[MAXK], ccount[MAXK];
    __shared__ unsigned char pa[MAXPAIR], pb[MAXPAIR];
    __shared__ int stop;

    const int F = xtr_row(B);
    const int F2 = 2 * F;
    const int BA = B + 1;
    const int npair = BA * (BA + 1) / 2;
    const int nb = mom_shape(B).nb;
    const int tid = threadIdx.x;
    uint16_t* XT = reinterpret_cast<uint16_t*>(dyn);                     // F2 x UPAD bf16
    float* Cs = reinterpret_cast<float*>(dyn + F2 * UPAD * 2);           // F2 x cs_stride(F2)

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
        const bool over = tot > static_cast<unsigned long long>(cap);
        stop = (dm->status != 0) || over;
        if (over && blockIdx.x == 0) atomicCAS(&dm->status, 0, CVA_ERR_CAPACITY);
    }
    build_pairs(pa, pb, BA);
    __syncthreads();
    if (stop) return;

    unsigned long long acc[3] = {0ull, 0ull, 0ull};
    int cur_class = -1;
    const unsigned int nunits = ustart[K];
    for (unsigned int u = blockIdx.x; u < nunits; u += gridDim.x) {
        int c = 0;
        while (u >= ustart[c + 1]) ++c;
        if (c != cur_class) {
            if (cur_class >= 0) moments_flush(dm, cur_class, nb, npair, pa, pb, acc);
            cur_class = c;
        }
        const unsigned int row0 = cstart[c] + (u - ustart[c]) * UNIT;
        const int len = static_cast<int>(min(static_cast<unsigned int>(UNIT), cstart[c] + ccount[c] - row0));
        gather_stage<NBAND>(XT, cube, B, P, list + static_cast<long long>(c) * cap + (row0 - cstart[c]),
                            xtr + static_cast<long long>(row0) * F, F, len);
        __syncthreads();
        moments_gram(XT, Cs, F, npair, pa, pb, acc);
    }
    if (cur_class >= 0) moments_flush(dm, cur_class, nb, npair, pa, pb, acc);
}

// ---------------------------------------------------------------------------
// Batched form: the same passes over the flattened work of many pages.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(TPB) kb_tile_count(const PageDev* __restrict__ pages, const int* __restrict__ tile_page)
{
    const int p = tile_page[blockIdx.x];
    const PageDev& pg = pages[p];
    // the training capacity is checked by the pool scan, over the whole batch
    tile_count_body(pg.labels, pg.P, pg.K, pg.B, pg.vec, 0x7FFFFFFFFFFFFFFFll, pg.ntiles, pg.tiles, pg.dm,
                    static_cast<int>(blockIdx.x - pg.tile0));
}

__global__ void __launch_bounds__(TPB)
kb_tile_compact(const PageDev* __restrict__ pages, const int* __restrict__ tile_page,
                unsigned int* __restrict__ list_pool)
{
    const int p = tile_page[blockIdx.x];
    const PageDev& pg = pages[p];
    if (pg.dm->status != 0) return;
    tile_compact_body(pg.labels, pg.P, pg.K, pg.vec, pg.tiles, pg.dm->cls_count, list_pool + pg.row0,
                      static_cast<int>(blockIdx.x - pg.tile0));
}

// Moment units of all pages: a unit is up to 256 rows of one class of one
// page, gathered from the page's cube and staged as in k_gather_moments (the
// rows also go to the pooled training matrix, which the training-range pass
// reads).  A CTA keeps its sums in registers while it stays on one (page,
// class) and merges them into that page's model when it moves on.  NBAND (24
// or MAXB) bounds the batch's band counts.
template <int NBAND>
__global__ void __launch_bounds__(TPB, 4)
kb_gather_moments(const PageDev* __restrict__ pages, int n, const BatchTotals* __restrict__ tot,
                  const unsigned int* __restrict__ list_pool, uint16_t* __restrict__ xtr_pool, int max_f)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned char pa[MAXPAIR], pb[MAXPAIR];
    __shared__ int s_page, s_class, s_len, s_skip;
    __shared__ unsigned int s_row0;
    const int tid = threadIdx.x;
    uint16_t* XT = reinterpret_cast<uint16_t*>(dyn);                          // (2 max_f) x UPAD bf16
    float* Cs = reinterpret_cast<float*>(dyn + 2 * max_f * UPAD * 2);         // Gram, row stride cs_stride

    unsigned long long acc[3] = {0ull, 0ull, 0ull};
    int cur_page = -1, cur_class = -1, cur_b = -1;
    // each CTA takes a contiguous run of units, so it seldom changes page or class
    const unsigned long long nunits = tot->units;
    const unsigned long long per = (nunits + gridDim.x - 1) / gridDim.x;
    const unsigned long long u_end = min(nunits, (blockIdx.x + 1ull) * per);
    // thread 0 keeps the current class's unit range and looks the page and
    // class up again only when a unit leaves it
    int c_page = -1, c_class = 0, c_skip = 1;
    unsigned long long c_u0 = 0, c_u1 = 0;
    unsigned int c_row = 0, c_nc = 0;
    for (unsigned long long u = blockIdx.x * per; u < u_end; ++u) {
        if (tid == 0) {
            if (c_page < 0 || u < c_u0 || u >= c_u1) {
                const int p = find_page(pages, n, u, [](const PageDev& q) { return q.unit0; });
                const PageDev& pg = pages[p];
                unsigned long long lu = u - pg.unit0;
                unsigned int row = 0, nc = 0;
                int c = 0;
                for (; c < pg.K; ++c) {
                    nc = pg.dm->cls_count[c];
                    const unsigned long long nu = (nc + UNIT - 1) / UNIT;
                    if (lu < nu) break;
                    lu -= nu;
                    row += nc;
                }
                c_page = p;
                c_class = c;
                c_skip = pg.dm->status != 0 || c >= pg.K;
                c_u0 = u - lu;
                c_u1 = c >= pg.K ? u + 1 : c_u0 + (nc + UNIT - 1) / UNIT;
                c_row = row;
                c_nc = c >= pg.K ? 0u : nc;
            }
            const unsigned int row0 = c_row + static_cast<unsigned int>(u - c_u0) * UNIT;
            s_page = c_page;
            s_class = c_class;
            s_row0 = row0;
            s_len = c_skip ? 0 : static_cast<int>(min(static_cast<unsigned int>(UNIT), c_row + c_nc - row0));
            s_skip = c_skip;
        }
        __syncthreads();
        const int p = s_page, c = s_class;
        const PageDev& pg = pages[p];
        const int B = pg.B, BA = B + 1;
        const int npair = BA * (BA + 1) / 2;
        if (p != cur_page || c != cur_class) {
            if (cur_page >= 0) moments_flush(pages[cur_page].dm, cur_class, mom_shape(cur_b).nb, (cur_b + 1) * (cur_b + 2) / 2,
                                             pa, pb, acc);
            if (B != cur_b) {
                __syncthreads();  // flush read the old tables
                build_pairs(pa, pb, BA);
                __syncthreads();
            }
            cur_page = p;
            cur_class = c;
            cur_b = B;
        }
        if (!s_skip) {
            const int F = xtr_row(B);
            gather_stage<NBAND>(XT, pg.cube, B, pg.P, list_pool + pg.row0 + s_row0,
                                xtr_pool + pg.xoff + static_cast<long long>(s_row0) * F, F, s_len);
            __syncthreads();
            moments_gram(XT, Cs, F, npair, pa, pb, acc);
        } else {
            __syncthreads();
        }
    }
    if (cur_page >= 0)
        moments_flush(pages[cur_page].dm, cur_class, mom_shape(cur_b).nb, (cur_b + 1) * (cur_b + 2) / 2, pa, pb, acc);
}

// ---------------------------------------------------------------------------
// Principal components (Section 2: the unsupervised PCA of the page): exact
// moments of the augmented vectors (x, 1) of every selected pixel, straight
// from the band-sequential cube, into class 0 of the model.  A unit is 256
// consecutive pixels: with 16-byte-aligned rows each warp stages band rows
// (8 pixels a lane, one 16-byte load), otherwise each thread stages one
// pixel.  Masked-out pixels stage as zero columns and add nothing.
// ---------------------------------------------------------------------------
__device__ inline uint32_t pack_bf16_pair(uint32_t a, uint32_t b)
{
    return bf16_of_byte(a) | (bf16_of_byte(b) << 16);
}

__global__ void __launch_bounds__(TPB)
k_pca_moments(const uint16_t* __restrict__ cube, int B, long long P, const uint8_t* __restrict__ mask, int vec,
              DevModel* __restrict__ dm)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ unsigned char pa[MAXPAIR], pb[MAXPAIR];
    const int F = xtr_row(B), BA = B + 1;
    const int npair = BA * (BA + 1) / 2;
    const int nb = mom_shape(B).nb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint16_t* XT = reinterpret_cast<uint16_t*>(dyn);
    float* Cs = reinterpret_cast<float*>(dyn + 2 * F * UPAD * 2);
    build_pairs(pa, pb, BA);
    __syncthreads();
    unsigned long long acc[3] = {0ull, 0ull, 0ull};
    const long long nunits = (P + UNIT - 1) / UNIT;
    const long long per = (nunits + gridDim.x - 1) / gridDim.x;
    const long long u0 = static_cast<long long>(blockIdx.x) * per;
    const long long u1 = u0 + per < nunits ? u0 + per : nunits;
    if (vec) {
        // software pipeline: the 16-byte band loads of unit u + 1 are issued
        // before the Gram matrix of unit u is formed
        constexpr int ROWS = (MAXB + 8 + NW - 1) / NW;  // rows f = warp + r NW a warp stages: 5 cover F <= 40
        uint4 nx[ROWS];
        uint32_t nsel = 0u;
        auto load_unit = [&](long long u) {
            const long long pl = u * UNIT + lane * 8;
            const bool in = pl < P;  // P % 8 == 0: whole groups of 8
            nsel = in ? 0xFFu : 0u;  // bit i: pixel pl + i selected
            if (in && mask) {
                const uint2 mv = *reinterpret_cast<const uint2*>(mask + pl);
                nsel = 0u;
                #pragma unroll
                for (int i = 0; i < 8; ++i) nsel |= ((((i < 4 ? mv.x : mv.y) >> (8 * (i & 3))) & 0xFFu) != 0u) << i;
            }
            #pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int f = warp + r * NW;
                nx[r] = make_uint4(0u, 0u, 0u, 0u);
                if (in && f < B) nx[r] = __ldcs(reinterpret_cast<const uint4*>(cube + static_cast<long long>(f) * P + pl));
            }
        };
        if (u0 < u1) load_unit(u0);
        for (long long u = u0; u < u1; ++u) {
            #pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const int f = warp + r * NW;
                if (f >= F) break;
                uint32_t x[8];
                if (f < B) {
                    const uint32_t wv[4] = {nx[r].x, nx[r].y, nx[r].z, nx[r].w};
                    #pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = ((nsel >> i) & 1u) ? ((wv[i >> 1] >> (16 * (i & 1))) & 0xFFFFu) : 0u;
                } else {
                    #pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = (f == B) ? ((nsel >> i) & 1u) : 0u;
                }
                const uint4 hi = make_uint4(pack_bf16_pair(x[0] >> 8, x[1] >> 8), pack_bf16_pair(x[2] >> 8, x[3] >> 8),
                                            pack_bf16_pair(x[4] >> 8, x[5] >> 8), pack_bf16_pair(x[6] >> 8, x[7] >> 8));
                const uint4 lo = make_uint4(pack_bf16_pair(x[0] & 0xFFu, x[1] & 0xFFu),
                                            pack_bf16_pair(x[2] & 0xFFu, x[3] & 0xFFu),
                                            pack_bf16_pair(x[4] & 0xFFu, x[5] & 0xFFu),
                                            pack_bf16_pair(x[6] & 0xFFu, x[7] & 0xFFu));
                *reinterpret_cast<uint4*>(XT + f * UPAD + lane * 8) = hi;
                *reinterpret_cast<uint4*>(XT + (F + f) * UPAD + lane * 8) = lo;
            }
            __syncthreads();
            if (u + 1 < u1) load_unit(u + 1);
            moments_gram(XT, Cs, F, npair, pa, pb, acc);
        }
    } else {
        for (long long u = u0; u < u1; ++u) {
            const long long p0 = u * UNIT;
            const long long p = p0 + tid;
            const bool sel = p < P && (!mask || mask[p] != 0);
            for (int f = 0; f < F; ++f) {
                uint32_t x = 0u;
                if (sel) x = f < B ? static_cast<uint32_t>(cube[static_cast<long long>(f) * P + p]) : (f == B ? 1u : 0u);
                XT[f * UPAD + tid] = static_cast<uint16_t>(bf16_of_byte(x >> 8));
                XT[(F + f) * UPAD + tid] = static_cast<uint16_t>(bf16_of_byte(x & 0xFFu));
            }
            __syncthreads();
            moments_gram(XT, Cs, F, npair, pa, pb, acc);
        }
    }
    moments_flush(dm, 0, nb, npair, pa, pb, acc);
}

// The exact moments of every class as a flat array: class c, then the upper
// triangle a <= b of the (B+1) x (B+1) augmented moment matrix in row-major
// order (entry (a, b) at c W + a (B+1) - a (a-1)/2 + (b - a), W = (B+1)(B+2)/2).
__global__ void k_moments_export(const DevModel* __restrict__ dm, int B, int K, long long* __restrict__ out)
{
    const int BA = B + 1, per = BA * (BA + 1) / 2;
    const int nb = mom_shape(B).nb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * per; i += gridDim.x * blockDim.x) {
        const int c = i / per;
        int q = i - c * per, a = 0;
        while (q >= BA - a) { q -= BA - a; ++a; }
        const int b = a + q;
        out[i] = static_cast<long long>(dm->mom[c][blk_index(a >> 2, b >> 2, nb)][(a & 3) * 4 + (b & 3)]);
    }
}

// The inverse: the given moments replace the model's (the entries outside
// the augmented matrix are not read by the finalize).
__global__ void k_moments_import(DevModel* __restrict__ dm, int B, int K, const long long* __restrict__ in)
{
    const int BA = B + 1, per = BA * (BA + 1) / 2;
    const int nb = mom_shape(B).nb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * per; i += gridDim.x * blockDim.x) {
        const int c = i / per;
        int q = i - c * per, a = 0;
        while (q >= BA - a) { q -= BA - a; ++a; }
        const int b = a + q;
        dm->mom[c][blk_index(a >> 2, b >> 2, nb)][(a & 3) * 4 + (b & 3)] = static_cast<unsigned long long>(in[i]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) dm->fitted = 0;
}

// ---------------------------------------------------------------------------
// Principal components, register form (B + 1 <= 24 augmented bands, P % 8 ==
// 0, 16-byte aligned cube, 8-byte aligned mask).  Each warp takes a
// contiguous range of pixels and forms the Gram matrix of the byte-split
// augmented vectors X = [h ; l] (2F rows: the high bytes of bands 0..F-1,
// then the low bytes; row B is the "1" of the augmented vector) with
// mma.sync m16n8k16 f16 x f16 -> f32, straight from its loads:
//   * the Gram matrix sums over pixels, so which pixel feeds which k slot of
//     an mma is free; lane (g, t) = (lane / 4, lane % 4) takes 8 consecutive
//     pixels of every 32 from one 16-byte load per band and feeds them to the
//     k slots it owns in the A fragment, and the B fragment of column group j
//     (columns = rows of X) is the A fragment's registers of row group j;
//   * lane g holds bands g, g + 8, g + 16 of each pixel: one 16-byte load per
//     band and 32 pixels, 64 contiguous bytes for the 4 lanes of a band;
//   * a byte v becomes the f16 value v exactly by one byte permute (the f16
//     bits of 1024 + v are 0x64 : v) and one packed f16 subtraction of 1024;
//   * each product is at most 255^2, so an FP32 accumulator stays an exact
//     integer (below 2^24) for 256 pixels; the warp drains its accumulators
//     into 32-bit integer sums every 256 pixels and into shared memory every
//     32768 (the 32-bit sums stay below 2^32), so no block barrier is taken
//     while pixels stream;
//   * at the end the CTA's 64-bit sums in shared memory are recombined into
//     moments, M = 65536 C_hh + 256 (C_hl + C_lh) + C_ll, and added to the
//     model with one atomic per moment.
// Only Gram tiles on or above the diagonal are formed: 12 mma per 16 pixels
// at F = 24.
// ---------------------------------------------------------------------------
namespace pcar {

constexpr int TPBR = 384;             // 12 warps, one CTA an SM
constexpr int DSTEP = 32;             // pixels of one double step (two mma k steps)
constexpr int DRAIN = 8;              // double steps between drains (256 pixels)
constexpr int FLUSH = 1024;           // double steps between flushes to shared memory (32768 pixels)

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                              uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// f16x2 of the low (hi = false) or high bytes of the two 16-bit values in w,
// exactly: the permute builds the f16 bit patterns of 1024 + byte, the
// packed subtraction removes 1024.
__device__ __forceinline__ uint32_t bytes_to_f16x2(uint32_t w, bool hi)
{
    const uint32_t biased = __byte_perm(w, 0x64646464u, hi ? 0x4341u : 0x4240u);
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(biased), "r"(0x64006400u));
    return r;
}

// Number of Gram tiles (16-row block R, 8-column group C) on or above the
// diagonal: C >= 2 R.
__host__ __device__ constexpr int ntiles(int F)
{
    return (2 * F / 16) * (2 * F / 8) - (2 * F / 16) * (2 * F / 16 - 1);
}

// The lane's 16-byte loads of one double step: bands g + 8 i < B from the
// cube, the "1" of the augmented vector as the value 1 at every pixel (its
// high byte 0, its low byte 1), padding bands 0; lanes past the warp's range
// load zeros.  With a mask, the values of pixels outside it become 0 (the
// "1" included), so they add nothing.
template <int NBL, bool MASKED>
__device__ __forceinline__ void load_dstep(const uint16_t* __restrict__ cube, const uint8_t* __restrict__ mask, int B,
                                           long long P, long long p, long long p_end, int g, uint4 (&v)[NBL])
{
    const bool in = p < p_end;
    #pragma unroll
    for (int i = 0; i < NBL; ++i) {
        const int band = g + 8 * i;
        v[i] = make_uint4(0u, 0u, 0u, 0u);
        if (in && band < B) v[i] = __ldcs(reinterpret_cast<const uint4*>(cube + static_cast<long long>(band) * P + p));
        else if (in && band == B) v[i] = make_uint4(0x00010001u, 0x00010001u, 0x00010001u, 0x00010001u);
    }
    if (MASKED && in) {
        const uint2 mv = *reinterpret_cast<const uint2*>(mask + p);
        // keep-mask of the two 16-bit values of word w (mask bytes 2 w, 2 w + 1)
        uint32_t keep[4];
        #pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t m = w < 2 ? mv.x : mv.y;
            const int j = 2 * (w & 1);
            keep[w] = (((m >> (8 * j)) & 0xFFu) ? 0x0000FFFFu : 0u) | (((m >> (8 * (j + 1))) & 0xFFu) ? 0xFFFF0000u : 0u);
        }
        #pragma unroll
        for (int i = 0; i < NBL; ++i) {
            v[i].x &= keep[0];
            v[i].y &= keep[1];
            v[i].z &= keep[2];
            v[i].w &= keep[3];
        }
    }
}

// Dynamic shared memory of k_pca_moments_reg<F>: the CTA's 64-bit Gram sums
// (2F x 2F) and every lane's 32-bit partial sums (NT x 4 a lane).
__host__ __device__ constexpr size_t reg_smem_bytes(int F)
{
    return static_cast<size_t>(2 * F) * (2 * F) * 8 + static_cast<size_t>(TPBR / 32) * ntiles(F) * 4 * 32 * 4;
}

template <int F, bool MASKED>
__global__ void __launch_bounds__(pcar::TPBR, 1)
k_pca_moments_reg(const uint16_t* __restrict__ cube, int B, long long P, const uint8_t* __restrict__ mask,
                  long long chunk, DevModel* __restrict__ dm)
{
    constexpr int NBL = F / 8;              // bands per lane
    constexpr int RB = 2 * F / 16;          // 16-row blocks of the Gram matrix
    constexpr int CG = 2 * F / 8;           // 8-column groups
    constexpr int NT = pcar::ntiles(F);
    constexpr int D = 4;                    // double steps in the load ring (three ahead)
    extern __shared__ __align__(16) unsigned char rdyn[];
    unsigned long long (*S)[2 * F] = reinterpret_cast<unsigned long long (*)[2 * F]>(rdyn);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
    // this lane's 32-bit sums: entry (q, e) at SS[(q * 4 + e) * 32 + lane] (one bank a lane)
    uint32_t* SS = reinterpret_cast<uint32_t*>(rdyn + static_cast<size_t>(2 * F) * (2 * F) * 8) +
                   static_cast<size_t>(warp) * NT * 4 * 32;
    for (int i = tid; i < 4 * F * F; i += pcar::TPBR) (&S[0][0])[i] = 0ull;
    for (int i = lane; i < NT * 4 * 32; i += 32) SS[i] = 0u;
    __syncthreads();

    const long long wid = (static_cast<long long>(blockIdx.x) * pcar::TPBR + tid) >> 5;
    const long long p_begin = wid * chunk;
    const long long p_end = min(P, p_begin + chunk);
    float acc[NT][4];
    #pragma unroll
    for (int q = 0; q < NT; ++q)
        #pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][e] = 0.0f;

    // FP32 accumulators (exact integers below 2^24) into the 32-bit sums
    auto drain = [&]() {
        #pragma unroll
        for (int q = 0; q < NT; ++q)
            #pragma unroll
            for (int e = 0; e < 4; ++e) {
                SS[(q * 4 + e) * 32 + lane] += __float2uint_rn(acc[q][e]);
                acc[q][e] = 0.0f;
            }
    };
    // 32-bit sums into the CTA's 64-bit sums; entry e of tile q of this lane
    // is row 16 R + g + 8 (e >> 1), column 8 C + 2 t + (e & 1)
    auto flush = [&]() {
        int q = 0;
        #pragma unroll
        for (int R = 0; R < RB; ++R)
            #pragma unroll
            for (int C = 2 * R; C < CG; ++C, ++q)
                #pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = 16 * R + g + 8 * (e >> 1), col = 8 * C + 2 * t + (e & 1);
                    uint32_t& v = SS[(q * 4 + e) * 32 + lane];
                    if (row <= col && v) atomicAdd(&S[row][col], static_cast<unsigned long long>(v));
                    v = 0u;
                }
    };
    auto compute = [&](const uint4 (&cur)[NBL]) {
        #pragma unroll
        for (int k = 0; k < 2; ++k) {
            // this k step: pixels 4 k .. 4 k + 3 of the lane's eight
            uint32_t X[2 * NBL][2];
            #pragma unroll
            for (int i = 0; i < NBL; ++i) {
                const uint32_t w0 = k ? cur[i].z : cur[i].x, w1 = k ? cur[i].w : cur[i].y;
                X[i][0] = pcar::bytes_to_f16x2(w0, true);
                X[i][1] = pcar::bytes_to_f16x2(w1, true);
                X[NBL + i][0] = pcar::bytes_to_f16x2(w0, false);
                X[NBL + i][1] = pcar::bytes_to_f16x2(w1, false);
            }
            int q = 0;
            #pragma unroll
            for (int R = 0; R < RB; ++R)
                #pragma unroll
                for (int C = 2 * R; C < CG; ++C, ++q)
                    pcar::mma_f16_16816(acc[q], X[2 * R][0], X[2 * R + 1][0], X[2 * R][1], X[2 * R + 1][1],
                                        X[C][0], X[C][1]);
        }
    };

    if (p_begin < p_end) {
        uint4 buf[D][NBL];
        #pragma unroll
        for (int j = 0; j < D - 1; ++j)
            load_dstep<NBL, MASKED>(cube, mask, B, P, p_begin + j * pcar::DSTEP + 8 * t, p_end, g, buf[j]);
        int rounds = 0;  // outer rounds of D double steps
        for (long long dp = p_begin; dp < p_end; dp += D * pcar::DSTEP) {
            #pragma unroll
            for (int j = 0; j < D; ++j) {
                // double steps past p_end load zeros and add nothing
                load_dstep<NBL, MASKED>(cube, mask, B, P, dp + (j + D - 1) * pcar::DSTEP + 8 * t, p_end, g,
                                        buf[(j + D - 1) % D]);
                compute(buf[j]);
            }
            ++rounds;
            if ((rounds * D) % pcar::DRAIN == 0) {
                drain();
                if ((rounds * D) % pcar::FLUSH == 0) flush();
            }
        }
        drain();
        flush();
    }
    __syncthreads();
    // moments of the augmented vectors: M[a][b] = 65536 hh + 256 (hl + lh) + ll
    const int BA = B + 1, nb = mom_shape(B).nb;
    for (int q = tid; q < BA * (BA + 1) / 2; q += pcar::TPBR) {
        int a = 0, r = q;
        while (r >= BA - a) { r -= BA - a; ++a; }
        const int b = a + r;
        const unsigned long long M = (S[a][b] << 16) + ((S[a][F + b] + S[b][F + a]) << 8) + S[F + a][F + b];
        if (M) atomicAdd(&dm->mom[0][blk_index(a >> 2, b >> 2, nb)][(a & 3) * 4 + (b & 3)], M);
    }
}

}  // namespace pcar

// Clears class 0's moments and the fit state before a principal-component fit.
__global__ void k_pca_reset(DevModel* __restrict__ dm, int B)
{
    const MomShape sh = mom_shape(B);
    for (int i = threadIdx.x; i < sh.nblk * 16; i += blockDim.x) dm->mom[0][i >> 4][i & 15] = 0ull;
    if (threadIdx.x == 0) {
        dm->status = CVA_OK;
        dm->fitted = 0;
    }
}

}  // namespace

cudaError_t launch_fit_moments(const uint16_t* cube, int B, long long P, const uint8_t* labels, int K,
                               DevModel* dm, uint16_t* xtr, unsigned int* list, long long cap, int num_sms,
                               cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(labels) % 16 == 0) ? 1 : 0;
    k_fit_reset<<<1, 256, 0, s>>>(dm, B, K);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_label_scan<<<static_cast<unsigned>(num_sms * 8), TPB, 0, s>>>(labels, P, K, vec, cap, list, dm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int F2 = 2 * xtr_row(B);
    const size_t smem = moments_smem_bytes(F2 / 2);
    // the unit count is only known on the device: one wave of resident CTAs
    // (five an SM up to 24 bands, ~36 KB of shared memory each), each taking
    // units in turn; CTAs without a unit exit at once
    if (B <= 24) {
        e = cudaFuncSetAttribute(k_gather_moments<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_gather_moments<24><<<static_cast<unsigned>(num_sms * gm_ctas(24)), TPB, smem, s>>>(cube, B, P, K, list, cap,
                                                                                               xtr, dm);
    } else {
        e = cudaFuncSetAttribute(k_gather_moments<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_gather_moments<MAXB><<<static_cast<unsigned>(num_sms * gm_ctas(MAXB)), TPB, smem, s>>>(cube, B, P, K, list,
                                                                                                   cap, xtr, dm);
    }
    return cudaGetLastError();
}

}  // namespace cva

namespace cva {

cudaError_t launch_batch_tile_count(const PageDev* pages, const int* tile_page, long long ntiles_total,
                                    cudaStream_t s)
{
    kb_tile_count<<<static_cast<unsigned>(ntiles_total), TPB, 0, s>>>(pages, tile_page);
    return cudaGetLastError();
}

cudaError_t launch_batch_tile_compact(const PageDev* pages, const int* tile_page, long long ntiles_total,
                                      unsigned int* list_pool, cudaStream_t s)
{
    kb_tile_compact<<<static_cast<unsigned>(ntiles_total), TPB, 0, s>>>(pages, tile_page, list_pool);
    return cudaGetLastError();
}

cudaError_t launch_batch_gather_moments(const PageDev* pages, int n, const BatchTotals* tot,
                                       const unsigned int* list_pool, uint16_t* xtr_pool, int max_b, int num_sms,
                                       cudaStream_t s)
{
    const int F = xtr_row(max_b);
    const size_t smem = moments_smem_bytes(F);
    cudaError_t e;
    if (max_b <= 24) {
        e = cudaFuncSetAttribute(kb_gather_moments<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        kb_gather_moments<24><<<static_cast<unsigned>(num_sms * 4), TPB, smem, s>>>(pages, n, tot, list_pool, xtr_pool, F);
    } else {
        e = cudaFuncSetAttribute(kb_gather_moments<MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        kb_gather_moments<MAXB><<<static_cast<unsigned>(num_sms * 4), TPB, smem, s>>>(pages, n, tot, list_pool, xtr_pool,
                                                                                       F);
    }
    return cudaGetLastError();
}

}  // namespace cva

namespace cva {

cudaError_t launch_moments_export(const DevModel* dm, int B, int K, long long* out, cudaStream_t s)
{
    k_moments_export<<<4, 256, 0, s>>>(dm, B, K, out);
    return cudaGetLastError();
}

cudaError_t launch_moments_import(DevModel* dm, int B, int K, const long long* in, cudaStream_t s)
{
    k_moments_import<<<4, 256, 0, s>>>(dm, B, K, in);
    return cudaGetLastError();
}

cudaError_t launch_pca_moments(const uint16_t* cube, int B, long long P, const uint8_t* mask, DevModel* dm,
                               int num_sms, cudaStream_t s)
{
    const int vec = (P % 8 == 0) && (reinterpret_cast<uintptr_t>(cube) % 16 == 0) &&
                    (!mask || reinterpret_cast<uintptr_t>(mask) % 8 == 0);
    const size_t smem = moments_smem_bytes(xtr_row(B));
    cudaError_t e = cudaFuncSetAttribute(k_pca_moments, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_pca_reset<<<1, 256, 0, s>>>(dm, B);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int F = xtr_row(B);
    const bool reg = F <= 24 && P % 8 == 0 && reinterpret_cast<uintptr_t>(cube) % 16 == 0 &&
                     (!mask || reinterpret_cast<uintptr_t>(mask) % 8 == 0);
    if (reg) {
        // one CTA of 12 warps an SM, each warp a contiguous run of pixels
        // (a multiple of 32, at least 256)
        const long long warps = static_cast<long long>(num_sms) * (pcar::TPBR / 32);
        long long chunk = (P + warps - 1) / warps;
        chunk = ((chunk + pcar::DSTEP - 1) / pcar::DSTEP) * pcar::DSTEP;
        if (chunk < 256) chunk = 256;
        const long long nw = (P + chunk - 1) / chunk;
        const unsigned grid = static_cast<unsigned>((nw + pcar::TPBR / 32 - 1) / (pcar::TPBR / 32));
        const size_t sm = pcar::reg_smem_bytes(F);
        auto go = [&](auto kern) -> cudaError_t {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
            if (e2 != cudaSuccess) return e2;
            kern<<<grid, pcar::TPBR, sm, s>>>(cube, B, P, mask, chunk, dm);
            return cudaGetLastError();
        };
        if (mask) {
            if (F == 8) return go(pcar::k_pca_moments_reg<8, true>);
            if (F == 16) return go(pcar::k_pca_moments_reg<16, true>);
            return go(pcar::k_pca_moments_reg<24, true>);
        }
        if (F == 8) return go(pcar::k_pca_moments_reg<8, false>);
        if (F == 16) return go(pcar::k_pca_moments_reg<16, false>);
        return go(pcar::k_pca_moments_reg<24, false>);
    }
    const long long units = (P + UNIT - 1) / UNIT;
    long long grid = static_cast<long long>(num_sms) * 6;
    if (grid > units) grid = units;
    k_pca_moments<<<static_cast<unsigned>(grid), TPB, smem, s>>>(cube, B, P, mask, vec, dm);
    return cudaGetLastError();
}

}  // namespace cva
