// project.cu -- projection of every pixel onto the canonical variates and the
// linear rescale of each projection to 8 bits.
//
// Section 2 of the paper multiplies the canonical coefficients with the band
// images, giving one floating-point image per variate, and maps each onto
// 0..255 either by its own range over all pixels or by the range of the
// training points' scores.  Here
//     y_j[p] = sum_b V[b][j] (x_b[p] - mu_b)
// is computed in FP32 as
//     y_j = sum_b Vf[b][j] ((2^23 + x_b) - (2^23 + m_b)) - d_j ,   m_b = rint(mu_b)
// where 2^23 + x_b is built by one byte permute (no integer-to-float
// conversion) and the subtraction is exact, so the centring costs nothing and
// loses nothing; d_j = sum_b V[b][j] (mu_b - m_b) is folded in once.  The
// 8-bit code is floor((y - lo) * 255 / (hi - lo) + 1/2) clamped to 0..255.
//
// The pass is bound by HBM bandwidth (2B bytes in, k or 4k bytes out per
// pixel).  The main kernel (k_project_v8) gives each thread 8 consecutive
// pixels, keeps 8 x k FP32 accumulators in registers, software-pipelines the
// 16-byte band loads in batches of 8 so that up to 256 bytes per thread are
// in flight, and writes 8-byte (u8) or 32-byte (f32) streaming stores.  Its
// twin k_project_r8 takes cubes whose bands do not start on 16-byte
// boundaries (P not a multiple of 8, or an unaligned cube) and unaligned
// outputs at the same traffic: two aligned 16-byte loads per band and group,
// funnel-shifted.  A scalar kernel is left for cubes of fewer than 32 pixels.
//
// The training-range kernel repeats the same FP32 operations, in the same
// order, on the training pixels, so that the extreme training pixels land on
// exactly 0 and 255 in the fused projection.  The batched kernels
// (kb_train_range, kb_project_v8) run the same per-pixel code over the
// flattened work of many pages (see batch.cu).
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int KCH = 8;   // variates per pass
constexpr int NWARP = TPB / 32;

template <int KV>
struct ProjSmem {
    float V[MAXB][KV];
    float shift[MAXB];
    float d[KV];
    float off[KV];
    float scale[KV];
    float mn[NWARP][KV];
    float mx[NWARP][KV];
};

template <int KV>
__device__ inline void load_coefs(ProjSmem<KV>& sm, const DevModel* dm, int B, int j0, int kc,
                                  const float* u8_range, bool u8)
{
    const int tid = threadIdx.x;
    for (int e = tid; e < MAXB * KV; e += TPB) {
        const int b = e / KV, j = e - (e / KV) * KV;
        sm.V[b][j] = (b < B && j < kc) ? dm->Vf[b][j0 + j] : 0.0f;
    }
    if (tid < MAXB) sm.shift[tid] = dm->shift[tid];
    if (tid < KV) {
        sm.d[tid] = tid < kc ? dm->dofs[j0 + tid] : 0.0f;
        float lo = 0.0f, hi = 0.0f;
        if (u8 && tid < kc) {
            lo = u8_range[2 * (j0 + tid)];
            hi = u8_range[2 * (j0 + tid) + 1];
        }
        const float sc = code_scale(lo, hi);
        sm.scale[tid] = sc;
        sm.off[tid] = code_offset(lo, sc);
    }
}

template <int KV>
__device__ inline void reduce_range(ProjSmem<KV>& sm, float (&mn)[KV], float (&mx)[KV], int kc,
                                    float* range_acc, int j0)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        float a = mn[j], b = mx[j];
        for (int o = 16; o > 0; o >>= 1) {
            a = fminf(a, __shfl_xor_sync(0xFFFFFFFFu, a, o));
            b = fmaxf(b, __shfl_xor_sync(0xFFFFFFFFu, b, o));
        }
        if (lane == 0) {
            sm.mn[warp][j] = a;
            sm.mx[warp][j] = b;
        }
    }
    __syncthreads();
    if (tid < kc) {
        float a = sm.mn[0][tid], b = sm.mx[0][tid];
        for (int w = 1; w < NWARP; ++w) {
            a = fminf(a, sm.mn[w][tid]);
            b = fmaxf(b, sm.mx[w][tid]);
        }
        atomic_min_float(range_acc + 2 * (j0 + tid), a);
        atomic_max_float(range_acc + 2 * (j0 + tid) + 1, b);
    }
}

// ---------------------------------------------------------------------------
// Register-pipelined streaming (P % 8 == 0, 16-byte aligned cube): each thread
// takes 8 consecutive pixels and walks the bands in batches of 8 rows, the
// 16-byte evict-first loads of the next batch issued before the current batch
// is computed, so up to 16 loads (256 bytes) per thread stay in flight while
// the coefficients in shared memory are reused for 8 pixels.
// ---------------------------------------------------------------------------
// Bands per pipelined batch of the ragged kernel (two batches in flight): 8
// up to 4 variates, 4 above, where 8 would spill the shuffled chunks (the
// aligned kernel keeps 8: measured, its few spilled words cost less than
// halving the bytes in flight).
__host__ __device__ constexpr int ragged_batch_bands(int KV) { return KV <= 4 ? 8 : 4; }

template <int KV>
__device__ inline void accumulate8(float (&acc)[KV][8], const uint4& w, const float* vrow, float shift)
{
    float x[8];
    x[0] = __fsub_rn(u16_lo_biased(w.x), shift);
    x[1] = __fsub_rn(u16_hi_biased(w.x), shift);
    x[2] = __fsub_rn(u16_lo_biased(w.y), shift);
    x[3] = __fsub_rn(u16_hi_biased(w.y), shift);
    x[4] = __fsub_rn(u16_lo_biased(w.z), shift);
    x[5] = __fsub_rn(u16_hi_biased(w.z), shift);
    x[6] = __fsub_rn(u16_lo_biased(w.w), shift);
    x[7] = __fsub_rn(u16_hi_biased(w.w), shift);
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        const float v = vrow[j];
        #pragma unroll
        for (int i = 0; i < 8; ++i) acc[j][i] = __fmaf_rn(v, x[i], acc[j][i]);
    }
}

// Pixels 8 g .. 8 g + 7 of one cube (plane = P / 8 groups per band): the
// pipelined band loads, the FP32 projection onto KV variates, and the stores.
// GUARD drops the outputs of variates kc .. KV-1 (batched pages with fewer
// variates than the launch).
template <int KV, bool F32, bool U8, bool RNG, bool GUARD>
__device__ __forceinline__ void project_group8(const uint16_t* __restrict__ cube, int B, long long P, long long g,
                                               const ProjSmem<KV>& sm, int j0, int kc, float* __restrict__ out_f32,
                                               uint8_t* __restrict__ out_u8, float (&mn)[KV], float (&mx)[KV])
{
    const long long plane = P / 8;  // band stride in uint4 units
    const uint4* src = reinterpret_cast<const uint4*>(cube) + g;
    constexpr int NB = 8;
    float acc[KV][8];
    #pragma unroll
    for (int j = 0; j < KV; ++j)
        #pragma unroll
        for (int i = 0; i < 8; ++i) acc[j][i] = 0.0f;
    uint4 wa[NB], wb[NB];
    #pragma unroll
    for (int u = 0; u < NB; ++u)
        if (u < B) wa[u] = __ldcs(src + u * plane);
    for (int b0 = 0;; b0 += 2 * NB) {
        // the batch tests are the same for every thread: whole batches are
        // skipped by branches, only a partial last batch is predicated
        const bool second = b0 + NB < B;
        if (second) {
            #pragma unroll
            for (int u = 0; u < NB; ++u)
                if (b0 + NB + u < B) wb[u] = __ldcs(src + (b0 + NB + u) * plane);
        }
        #pragma unroll
        for (int u = 0; u < NB; ++u)
            if (b0 + u < B) accumulate8<KV>(acc, wa[u], sm.V[b0 + u], sm.shift[b0 + u]);
        if (!second) break;
        const bool third = b0 + 2 * NB < B;
        if (third) {
            #pragma unroll
            for (int u = 0; u < NB; ++u)
                if (b0 + 2 * NB + u < B) wa[u] = __ldcs(src + (b0 + 2 * NB + u) * plane);
        }
        #pragma unroll
        for (int u = 0; u < NB; ++u)
            if (b0 + NB + u < B) accumulate8<KV>(acc, wb[u], sm.V[b0 + NB + u], sm.shift[b0 + NB + u]);
        if (!third) break;
    }
    const long long p = g * 8;
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        if (GUARD && j >= kc) break;
        float y[8];
        #pragma unroll
        for (int i = 0; i < 8; ++i) y[i] = __fsub_rn(acc[j][i], sm.d[j]);
        if (F32) {
            float4* dst = reinterpret_cast<float4*>(out_f32 + static_cast<long long>(j0 + j) * P + p);
            __stcs(dst, make_float4(y[0], y[1], y[2], y[3]));
            __stcs(dst + 1, make_float4(y[4], y[5], y[6], y[7]));
        }
        if (U8) {
            const float sc = sm.scale[j], of = sm.off[j];
            uint32_t c[8];
            #pragma unroll
            for (int i = 0; i < 8; ++i) c[i] = to_code(y[i], sc, of);
            const uint2 packed = make_uint2(c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24),
                                            c[4] | (c[5] << 8) | (c[6] << 16) | (c[7] << 24));
            __stcs(reinterpret_cast<uint2*>(out_u8 + static_cast<long long>(j0 + j) * P + p), packed);
        }
        if (RNG) {
            #pragma unroll
            for (int i = 0; i < 8; ++i) { mn[j] = fminf(mn[j], y[i]); mx[j] = fmaxf(mx[j], y[i]); }
        }
    }
}

template <int KV, bool F32, bool U8, bool RNG>
__global__ void __launch_bounds__(TPB, 2)
k_project_v8(const uint16_t* __restrict__ cube, int B, long long P, const DevModel* __restrict__ dm,
             int j0, const float* __restrict__ u8_range, float* __restrict__ out_f32,
             uint8_t* __restrict__ out_u8, float* __restrict__ range_acc)
{
    __shared__ ProjSmem<KV> sm;
    if (dm->status != 0 || !dm->fitted) return;
    load_coefs<KV>(sm, dm, B, j0, KV, u8_range, U8);
    __syncthreads();

    float mn[KV], mx[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) { mn[j] = __int_as_float(0x7F800000); mx[j] = __int_as_float(0xFF800000); }

    const long long ngroups = P / 8;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    for (long long g = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x; g < ngroups; g += stride)
        project_group8<KV, F32, U8, RNG, false>(cube, B, P, g, sm, j0, KV, out_f32, out_u8, mn, mx);
    if (RNG) reduce_range<KV>(sm, mn, mx, KV, range_acc, j0);
}

// ---------------------------------------------------------------------------
// Ragged cubes (P % 8 != 0, or a cube that does not start on 16 bytes): band
// b then starts sh[b] = (off + b P) mod 8 values into a 16-byte chunk of the
// cube (A: the cube's address rounded down to 16 bytes, off: the cube's
// offset from it in values), so the 8 values of a pixel group straddle two
// aligned chunks: each lane loads one chunk per band, takes the next from the
// neighbouring lane by a warp shuffle, and funnel-shifts the group's values
// out of the pair (a warp projects 31 groups from 32 chunks), so a band costs
// one 16-byte load per lane as in the aligned kernel.  Groups g in [g_lo, g_hi) keep every
// chunk inside the cube: g_lo = 1 when off > 0 (the first chunk of band 0
// starts before the cube), g_hi = floor((P - 15) / 8) (the second chunk of
// the last band stays before its end); the few pixels outside them are
// projected one per thread by the grid's last CTA.  Stores take the widest
// width the alignment of each output plane allows.
// ---------------------------------------------------------------------------
struct RaggedBands {
    long long c0[MAXB];  // chunk of A holding the first value of band b
    int sh[MAXB];        // values of that chunk before band b starts
};

// Values s .. s + 7 of the 16 values in lo, hi (s uniform across the warp).
__device__ __forceinline__ uint4 take8(const uint4& lo, const uint4& hi, int s)
{
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    const uint32_t bits = static_cast<uint32_t>(s & 1) * 16u;
    uint32_t r[4];
    switch (s >> 1) {
        case 0:
            #pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = __funnelshift_r(w[i], w[i + 1], bits);
            break;
        case 1:
            #pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = __funnelshift_r(w[i + 1], w[i + 2], bits);
            break;
        case 2:
            #pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = __funnelshift_r(w[i + 2], w[i + 3], bits);
            break;
        default:
            #pragma unroll
            for (int i = 0; i < 4; ++i) r[i] = __funnelshift_r(w[i + 3], w[i + 4], bits);
            break;
    }
    return make_uint4(r[0], r[1], r[2], r[3]);
}

// Store 8 consecutive bytes / floats at any alignment (the alignment is the
// same for every thread of a plane, so the branches do not diverge).
__device__ __forceinline__ void store8_u8(uint8_t* dst, uint32_t lo4, uint32_t hi4)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
    if ((a & 7) == 0) {
        __stcs(reinterpret_cast<uint2*>(dst), make_uint2(lo4, hi4));
    } else if ((a & 3) == 0) {
        __stcs(reinterpret_cast<unsigned int*>(dst), lo4);
        __stcs(reinterpret_cast<unsigned int*>(dst) + 1, hi4);
    } else if ((a & 1) == 0) {
        unsigned short* d = reinterpret_cast<unsigned short*>(dst);
        __stcs(d, static_cast<unsigned short>(lo4 & 0xFFFFu));
        __stcs(d + 1, static_cast<unsigned short>(lo4 >> 16));
        __stcs(d + 2, static_cast<unsigned short>(hi4 & 0xFFFFu));
        __stcs(d + 3, static_cast<unsigned short>(hi4 >> 16));
    } else {
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
            dst[i] = static_cast<uint8_t>(lo4 >> (8 * i));
            dst[4 + i] = static_cast<uint8_t>(hi4 >> (8 * i));
        }
    }
}

__device__ __forceinline__ void store8_f32(float* dst, const float (&y)[8])
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst);
    if ((a & 15) == 0) {
        __stcs(reinterpret_cast<float4*>(dst), make_float4(y[0], y[1], y[2], y[3]));
        __stcs(reinterpret_cast<float4*>(dst) + 1, make_float4(y[4], y[5], y[6], y[7]));
    } else if ((a & 7) == 0) {
        #pragma unroll
        for (int i = 0; i < 4; ++i) __stcs(reinterpret_cast<float2*>(dst) + i, make_float2(y[2 * i], y[2 * i + 1]));
    } else {
        #pragma unroll
        for (int i = 0; i < 8; ++i) __stcs(dst + i, y[i]);
    }
}

// 31 pixel groups gw .. gw + 30 of a ragged cube, one per lane of the warp:
// lane l loads chunk c0[b] + gw + l of every band (one 16-byte load), and the
// group of lane l < 31 takes its values from its own chunk and lane l + 1's
// (a warp shuffle), so every band costs one load per lane, pipelined in
// batches of 8 bands as in the aligned kernel.  Lanes past g_hi load the last
// in-bounds chunk (needed by the lane before them) and store nothing.  Every
// lane of the warp calls this with the same gw.
template <int KV, bool F32, bool U8, bool RNG>
__device__ __forceinline__ void project_warp_ragged(const uint4* __restrict__ A, const RaggedBands& rb, int B,
                                                    long long P, long long gw, long long g_hi,
                                                    const ProjSmem<KV>& sm, int j0, float* __restrict__ out_f32,
                                                    uint8_t* __restrict__ out_u8, float (&mn)[KV], float (&mx)[KV])
{
    const int lane = threadIdx.x & 31;
    const long long g = gw + lane;
    const long long gc = g <= g_hi ? g : g_hi;  // chunk offset of this lane's load (in bounds)
    const bool active = lane < 31 && g < g_hi;
    float acc[KV][8];
    #pragma unroll
    for (int j = 0; j < KV; ++j)
        #pragma unroll
        for (int i = 0; i < 8; ++i) acc[j][i] = 0.0f;
    auto take = [&](const uint4& lo, int b) -> uint4 {
        const int sh = rb.sh[b];
        if (!sh) return lo;  // the band starts on 16 bytes: the chunk is the group
        uint4 hi;
        hi.x = __shfl_down_sync(0xFFFFFFFFu, lo.x, 1);
        hi.y = __shfl_down_sync(0xFFFFFFFFu, lo.y, 1);
        hi.z = __shfl_down_sync(0xFFFFFFFFu, lo.z, 1);
        hi.w = __shfl_down_sync(0xFFFFFFFFu, lo.w, 1);
        return take8(lo, hi, sh);
    };
    constexpr int NB = ragged_batch_bands(KV);
    uint4 wa[NB], wb[NB];
    #pragma unroll
    for (int u = 0; u < NB; ++u)
        if (u < B) wa[u] = __ldcs(A + rb.c0[u] + gc);
    for (int b0 = 0;; b0 += 2 * NB) {
        const bool second = b0 + NB < B;
        if (second) {
            #pragma unroll
            for (int u = 0; u < NB; ++u)
                if (b0 + NB + u < B) wb[u] = __ldcs(A + rb.c0[b0 + NB + u] + gc);
        }
        #pragma unroll
        for (int u = 0; u < NB; ++u)
            if (b0 + u < B) accumulate8<KV>(acc, take(wa[u], b0 + u), sm.V[b0 + u], sm.shift[b0 + u]);
        if (!second) break;
        const bool third = b0 + 2 * NB < B;
        if (third) {
            #pragma unroll
            for (int u = 0; u < NB; ++u)
                if (b0 + 2 * NB + u < B) wa[u] = __ldcs(A + rb.c0[b0 + 2 * NB + u] + gc);
        }
        #pragma unroll
        for (int u = 0; u < NB; ++u)
            if (b0 + NB + u < B) accumulate8<KV>(acc, take(wb[u], b0 + NB + u), sm.V[b0 + NB + u], sm.shift[b0 + NB + u]);
        if (!third) break;
    }
    if (!active) return;
    const long long p = g * 8;
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        float y[8];
        #pragma unroll
        for (int i = 0; i < 8; ++i) y[i] = __fsub_rn(acc[j][i], sm.d[j]);
        if (F32) store8_f32(out_f32 + static_cast<long long>(j0 + j) * P + p, y);
        if (U8) {
            const float sc = sm.scale[j], of = sm.off[j];
            uint32_t c[8];
            #pragma unroll
            for (int i = 0; i < 8; ++i) c[i] = to_code(y[i], sc, of);
            store8_u8(out_u8 + static_cast<long long>(j0 + j) * P + p, c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24),
                      c[4] | (c[5] << 8) | (c[6] << 16) | (c[7] << 24));
        }
        if (RNG) {
            #pragma unroll
            for (int i = 0; i < 8; ++i) { mn[j] = fminf(mn[j], y[i]); mx[j] = fmaxf(mx[j], y[i]); }
        }
    }
}

// One pixel, any alignment (the scalar kernel's arithmetic, in the same order).
template <int KV, bool F32, bool U8, bool RNG>
__device__ __forceinline__ void project_pixel(const uint16_t* __restrict__ cube, int B, long long P, long long p,
                                              const ProjSmem<KV>& sm, int j0, int kc, float* __restrict__ out_f32,
                                              uint8_t* __restrict__ out_u8, float (&mn)[KV], float (&mx)[KV])
{
    float acc[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) acc[j] = 0.0f;
    for (int b = 0; b < B; ++b) {
        const uint32_t x = __ldcs(cube + static_cast<long long>(b) * P + p);
        const float xs = __fsub_rn(u16_biased(x), sm.shift[b]);
        #pragma unroll
        for (int j = 0; j < KV; ++j) acc[j] = __fmaf_rn(sm.V[b][j], xs, acc[j]);
    }
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        if (j >= kc) break;
        const float y = __fsub_rn(acc[j], sm.d[j]);
        if (F32) out_f32[static_cast<long long>(j0 + j) * P + p] = y;
        if (U8) out_u8[static_cast<long long>(j0 + j) * P + p] = static_cast<uint8_t>(to_code(y, sm.scale[j], sm.off[j]));
        if (RNG) { mn[j] = fminf(mn[j], y); mx[j] = fmaxf(mx[j], y); }
    }
}

template <int KV, bool F32, bool U8, bool RNG>
__global__ void __launch_bounds__(TPB, 2)
k_project_r8(const uint16_t* __restrict__ cube, int B, long long P, long long g_lo, long long g_hi,
             const DevModel* __restrict__ dm, int j0, const float* __restrict__ u8_range,
             float* __restrict__ out_f32, uint8_t* __restrict__ out_u8, float* __restrict__ range_acc)
{
    __shared__ ProjSmem<KV> sm;
    __shared__ RaggedBands rb;
    if (dm->status != 0 || !dm->fitted) return;
    load_coefs<KV>(sm, dm, B, j0, KV, u8_range, U8);
    const uintptr_t addr = reinterpret_cast<uintptr_t>(cube);
    const uint4* A = reinterpret_cast<const uint4*>(addr & ~static_cast<uintptr_t>(15));
    const long long off = static_cast<long long>((addr & 15) >> 1);
    if (threadIdx.x < MAXB) {
        const long long e = off + static_cast<long long>(threadIdx.x) * P;
        rb.c0[threadIdx.x] = e >> 3;
        rb.sh[threadIdx.x] = static_cast<int>(e & 7);
    }
    __syncthreads();

    float mn[KV], mx[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) { mn[j] = __int_as_float(0x7F800000); mx[j] = __int_as_float(0xFF800000); }
    // warp w takes groups g_lo + 31 w .. + 30, then strides over the grid's warps
    const long long wid = (static_cast<long long>(blockIdx.x) * TPB + threadIdx.x) >> 5;
    const long long nwarps = (static_cast<long long>(gridDim.x) * TPB) >> 5;
    for (long long gw = g_lo + 31 * wid; gw < g_hi; gw += 31 * nwarps)
        project_warp_ragged<KV, F32, U8, RNG>(A, rb, B, P, gw, g_hi, sm, j0, out_f32, out_u8, mn, mx);
    // the pixels outside the groups: [0, 8 g_lo) and [8 g_hi, P), fewer than 32
    if (blockIdx.x == gridDim.x - 1) {
        const long long head = 8 * g_lo, tail0 = 8 * g_hi;
        const long long n = head + (P - tail0);
        for (long long t = threadIdx.x; t < n; t += TPB) {
            const long long p = t < head ? t : tail0 + (t - head);
            project_pixel<KV, F32, U8, RNG>(cube, B, P, p, sm, j0, KV, out_f32, out_u8, mn, mx);
        }
    }
    if (RNG) reduce_range<KV>(sm, mn, mx, KV, range_acc, j0);
}

// Scalar path: pixels [p_begin, P), one pixel per thread per step, any alignment.
template <bool F32, bool U8, bool RNG>
__global__ void __launch_bounds__(TPB)
k_project_s(const uint16_t* __restrict__ cube, int B, long long P, long long p_begin,
            const DevModel* __restrict__ dm, int j0, int kc, const float* __restrict__ u8_range,
            float* __restrict__ out_f32, uint8_t* __restrict__ out_u8, float* __restrict__ range_acc)
{
    __shared__ ProjSmem<KCH> sm;
    if (dm->status != 0 || !dm->fitted) return;
    load_coefs<KCH>(sm, dm, B, j0, kc, u8_range, U8);
    __syncthreads();
    float mn[KCH], mx[KCH];
    #pragma unroll
    for (int j = 0; j < KCH; ++j) { mn[j] = __int_as_float(0x7F800000); mx[j] = __int_as_float(0xFF800000); }
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    for (long long p = p_begin + static_cast<long long>(blockIdx.x) * TPB + threadIdx.x; p < P; p += stride) {
        float acc[KCH];
        #pragma unroll
        for (int j = 0; j < KCH; ++j) acc[j] = 0.0f;
        for (int b = 0; b < B; ++b) {
            const uint32_t x = __ldcs(cube + static_cast<long long>(b) * P + p);
            const float xs = __fsub_rn(u16_biased(x), sm.shift[b]);
            #pragma unroll
            for (int j = 0; j < KCH; ++j) acc[j] = __fmaf_rn(sm.V[b][j], xs, acc[j]);
        }
        #pragma unroll
        for (int j = 0; j < KCH; ++j) {
            if (j >= kc) break;
            const float y = __fsub_rn(acc[j], sm.d[j]);
            if (F32) out_f32[static_cast<long long>(j0 + j) * P + p] = y;
            if (U8) out_u8[static_cast<long long>(j0 + j) * P + p] = static_cast<uint8_t>(to_code(y, sm.scale[j], sm.off[j]));
            if (RNG) { mn[j] = fminf(mn[j], y); mx[j] = fmaxf(mx[j], y); }
        }
    }
    if (RNG) reduce_range<KCH>(sm, mn, mx, kc, range_acc, j0);
}

// Training-score range of variates [j0, j0 + kc): same FP32 operations as the
// projection, on the rows of the gathered training matrix (x_0 .. x_{B-1}, 1, 0 ..).
template <int KV>
__device__ __forceinline__ void train_row(const ProjSmem<KV>& sm, const uint16_t* __restrict__ xrow, int B, int BR,
                                          float (&mn)[KV], float (&mx)[KV])
{
    const uint4* row = reinterpret_cast<const uint4*>(xrow);
    uint32_t pk[(MAXB + 8) / 2];
    #pragma unroll
    for (int q = 0; q < (MAXB + 8) / 8; ++q) {
        if (q * 8 < BR) {
            const uint4 v = __ldg(row + q);
            pk[4 * q] = v.x; pk[4 * q + 1] = v.y; pk[4 * q + 2] = v.z; pk[4 * q + 3] = v.w;
        } else {
            pk[4 * q] = pk[4 * q + 1] = pk[4 * q + 2] = pk[4 * q + 3] = 0u;
        }
    }
    float acc[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) acc[j] = 0.0f;
    #pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        if (b < B) {
            const uint32_t w = pk[b >> 1];
            const float xs = __fsub_rn((b & 1) ? u16_hi_biased(w) : u16_lo_biased(w), sm.shift[b]);
            #pragma unroll
            for (int j = 0; j < KV; ++j) acc[j] = __fmaf_rn(sm.V[b][j], xs, acc[j]);
        }
    }
    #pragma unroll
    for (int j = 0; j < KV; ++j) {
        const float y = __fsub_rn(acc[j], sm.d[j]);
        mn[j] = fminf(mn[j], y);
        mx[j] = fmaxf(mx[j], y);
    }
}

template <int KV>
__global__ void __launch_bounds__(TPB)
k_train_range(int B, int K, const uint16_t* __restrict__ xtr, DevModel* __restrict__ dm, int j0)
{
    __shared__ ProjSmem<KV> sm;
    if (dm->status != 0 || !dm->fitted) return;
    load_coefs<KV>(sm, dm, B, j0, KV, nullptr, false);
    __syncthreads();
    unsigned int N = 0;
    for (int c = 0; c < K; ++c) N += dm->cls_count[c];
    const int BR = xtr_row(B);
    float mn[KV], mx[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) { mn[j] = __int_as_float(0x7F800000); mx[j] = __int_as_float(0xFF800000); }
    const unsigned int stride = gridDim.x * TPB;
    for (unsigned int i = blockIdx.x * TPB + threadIdx.x; i < N; i += stride)
        train_row<KV>(sm, xtr + static_cast<long long>(i) * BR, B, BR, mn, mx);
    reduce_range<KV>(sm, mn, mx, KV, dm->train_range, j0);
}

// ---------------------------------------------------------------------------
// Batched form.  Training-range items are 256 rows of one page; projection
// items are `gpi` groups of TPB x 8 pixels of one page.  A CTA walks its
// items in order and reloads the coefficients (and, for the range, merges
// its extremes) when the page changes; pages that failed are skipped.
// ---------------------------------------------------------------------------
template <int KV>
__global__ void __launch_bounds__(TPB)
kb_train_range(const PageDev* __restrict__ pages, int n, const BatchTotals* __restrict__ tot,
               const uint16_t* __restrict__ xtr_pool)
{
    __shared__ ProjSmem<KV> sm;
    float mn[KV], mx[KV];
    int cur = -1;
    // each CTA takes a contiguous run of items, so it seldom changes page
    const unsigned long long nitems = tot->titems;
    const unsigned long long per = (nitems + gridDim.x - 1) / gridDim.x;
    const unsigned long long it_end = min(nitems, (blockIdx.x + 1ull) * per);
    unsigned long long r0 = 0, r1 = 0;  // items of the current page
    int p = 0;
    for (unsigned long long it = blockIdx.x * per; it < it_end; ++it) {
        if (it < r0 || it >= r1) {
            p = find_page(pages, n, it, [](const PageDev& q) { return q.titem0; });
            r0 = pages[p].titem0;
            r1 = r0 + (pages[p].nrows + BATCH_ROWS_PER_ITEM - 1) / BATCH_ROWS_PER_ITEM;
            if (r1 <= it) r1 = it + 1;
        }
        const PageDev& pg = pages[p];
        if (pg.dm->status != 0 || !pg.dm->fitted) continue;
        if (p != cur) {
            if (cur >= 0) reduce_range<KV>(sm, mn, mx, pages[cur].k, pages[cur].dm->train_range, 0);
            __syncthreads();
            load_coefs<KV>(sm, pg.dm, pg.B, 0, pg.k, nullptr, false);
            __syncthreads();
            #pragma unroll
            for (int j = 0; j < KV; ++j) { mn[j] = __int_as_float(0x7F800000); mx[j] = __int_as_float(0xFF800000); }
            cur = p;
        }
        const unsigned long long i = (it - pg.titem0) * BATCH_ROWS_PER_ITEM + threadIdx.x;
        const int BR = xtr_row(pg.B);
        if (threadIdx.x < BATCH_ROWS_PER_ITEM && i < pg.nrows)
            train_row<KV>(sm, xtr_pool + pg.xoff + i * BR, pg.B, BR, mn, mx);
    }
    if (cur >= 0) reduce_range<KV>(sm, mn, mx, pages[cur].k, pages[cur].dm->train_range, 0);
}

template <int KV>
__global__ void __launch_bounds__(TPB, 2)
kb_project_v8(const PageDev* __restrict__ pages, const int* __restrict__ item_page, long long it_begin,
              long long it_end, int gpi, int contiguous)
{
    __shared__ ProjSmem<KV> sm;
    float mn[KV], mx[KV];
    int cur = -1;
    // persistent CTAs take contiguous runs of items (few page changes);
    // otherwise one CTA per item
    long long it0 = it_begin + blockIdx.x, it1 = it_end, step = gridDim.x;
    if (contiguous) {
        const long long nitems = it_end - it_begin;
        const long long per = (nitems + gridDim.x - 1) / gridDim.x;
        it0 = it_begin + static_cast<long long>(blockIdx.x) * per;
        it1 = it0 + per < it_end ? it0 + per : it_end;
        step = 1;
    }
    for (long long it = it0; it < it1; it += step) {
        const int p = item_page[it];
        const PageDev& pg = pages[p];
        if (pg.dm->status != 0 || !pg.dm->fitted) continue;
        if (p != cur) {
            __syncthreads();
            load_coefs<KV>(sm, pg.dm, pg.B, 0, pg.k, pg.dm->train_range, true);
            __syncthreads();
            cur = p;
        }
        const long long ngroups = pg.P / 8;
        const long long g0 = (it - pg.item0) * static_cast<long long>(gpi) * TPB + threadIdx.x;
        for (int r = 0; r < gpi; ++r) {
            const long long g = g0 + static_cast<long long>(r) * TPB;
            if (g < ngroups)
                project_group8<KV, false, true, false, true>(pg.cube, pg.B, pg.P, g, sm, 0, pg.k, nullptr, pg.out,
                                                             mn, mx);
        }
    }
}

__global__ void k_range_init(float* range, int k)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) {
        range[2 * j] = __int_as_float(0x7F800000);
        range[2 * j + 1] = __int_as_float(0xFF800000);
    }
}

// Range of FP32 projections (k x P), 4 pixels per thread where aligned.
__global__ void __launch_bounds__(TPB)
k_f32_range(const float* __restrict__ proj, int k, long long P, int vec, float* __restrict__ range_acc)
{
    __shared__ float smn[NWARP], smx[NWARP];
    const int j = blockIdx.y;
    const float* src = proj + static_cast<long long>(j) * P;
    float a = __int_as_float(0x7F800000), b = __int_as_float(0xFF800000);
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    const long long start = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = P / 4;
        for (long long g = start; g < n4; g += stride) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(src) + g);
            a = fminf(fminf(a, v.x), fminf(v.y, fminf(v.z, v.w)));
            b = fmaxf(fmaxf(b, v.x), fmaxf(v.y, fmaxf(v.z, v.w)));
        }
        done = n4 * 4;
    }
    for (long long p = done + start; p < P; p += stride) {
        const float v = src[p];
        a = fminf(a, v);
        b = fmaxf(b, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a = fminf(a, __shfl_xor_sync(0xFFFFFFFFu, a, o));
        b = fmaxf(b, __shfl_xor_sync(0xFFFFFFFFu, b, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { smn[warp] = a; smx[warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < NWARP; ++w) { a = fminf(a, smn[w]); b = fmaxf(b, smx[w]); }
        a = fminf(a, smn[0]);
        b = fmaxf(b, smx[0]);
        atomic_min_float(range_acc + 2 * j, a);
        atomic_max_float(range_acc + 2 * j + 1, b);
    }
}

// FP32 projections (k x P) to 8-bit codes with the range (lo, hi) pairs.
__global__ void __launch_bounds__(TPB)
k_f32_to_u8(const float* __restrict__ proj, int k, long long P, int vec, const float* __restrict__ range,
            uint8_t* __restrict__ out)
{
    const int j = blockIdx.y;
    const float sc = code_scale(range[2 * j], range[2 * j + 1]);
    const float lo = code_offset(range[2 * j], sc);  // the code offset
    const float* src = proj + static_cast<long long>(j) * P;
    uint8_t* dst = out + static_cast<long long>(j) * P;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    const long long start = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = P / 4;
        for (long long g = start; g < n4; g += stride) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(src) + g);
            const uint32_t c = to_code(v.x, sc, lo) | (to_code(v.y, sc, lo) << 8) |
                               (to_code(v.z, sc, lo) << 16) | (to_code(v.w, sc, lo) << 24);
            __stcs(reinterpret_cast<unsigned int*>(dst) + g, c);
        }
        done = n4 * 4;
    }
    for (long long p = done + start; p < P; p += stride) dst[p] = static_cast<uint8_t>(to_code(src[p], sc, lo));
}

template <int KV, bool F32, bool U8, bool RNG>
cudaError_t run_v8(const uint16_t* cube, int B, long long P, const DevModel* dm, int j0,
                   const float* u8_range, float* out_f32, uint8_t* out_u8, float* range_acc,
                   int num_sms, cudaStream_t s)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project_v8<KV, F32, U8, RNG>, TPB, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const long long ngroups = P / 8;
    long long grid = (ngroups + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_project_v8<KV, F32, U8, RNG><<<static_cast<unsigned>(grid), TPB, 0, s>>>(cube, B, P, dm, j0, u8_range,
                                                                           out_f32, out_u8, range_acc);
    return cudaGetLastError();
}

template <int KV, bool F32, bool U8, bool RNG>
cudaError_t run_r8(const uint16_t* cube, int B, long long P, const DevModel* dm, int j0,
                   const float* u8_range, float* out_f32, uint8_t* out_u8, float* range_acc,
                   int num_sms, cudaStream_t s)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project_r8<KV, F32, U8, RNG>, TPB, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const long long off = static_cast<long long>((reinterpret_cast<uintptr_t>(cube) & 15) >> 1);
    const long long g_lo = off > 0 ? 1 : 0;
    const long long g_hi = (P - 15) / 8;  // caller guarantees P >= 32
    const long long per_cta = 31LL * (TPB / 32);  // groups a CTA takes per round
    long long grid = (g_hi - g_lo + per_cta - 1) / per_cta;
    const long long cap = static_cast<long long>(num_sms) * per_sm;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_project_r8<KV, F32, U8, RNG><<<static_cast<unsigned>(grid), TPB, 0, s>>>(cube, B, P, g_lo, g_hi, dm, j0, u8_range,
                                                                           out_f32, out_u8, range_acc);
    return cudaGetLastError();
}

// The pixel-count limit below which the scalar kernel takes the whole cube.
constexpr long long RAGGED_MIN_P = 32;

template <bool F32, bool U8, bool RNG>
cudaError_t run_chunk(const uint16_t* cube, int B, long long P, const DevModel* dm, int j0, int kc,
                      const float* u8_range, float* out_f32, uint8_t* out_u8, float* range_acc,
                      bool vec, int num_sms, cudaStream_t s)
{
    long long p_tail = 0;
    if (!vec && P >= RAGGED_MIN_P) {
        switch (kc) {
            case 1: return run_r8<1, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 2: return run_r8<2, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 3: return run_r8<3, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 4: return run_r8<4, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 5: return run_r8<5, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 6: return run_r8<6, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            case 7: return run_r8<7, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
            default: return run_r8<8, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s);
        }
    }
    if (vec) {
        cudaError_t e = cudaSuccess;
        switch (kc) {
            case 1: e = run_v8<1, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 2: e = run_v8<2, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 3: e = run_v8<3, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 4: e = run_v8<4, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 5: e = run_v8<5, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 6: e = run_v8<6, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            case 7: e = run_v8<7, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
            default: e = run_v8<8, F32, U8, RNG>(cube, B, P, dm, j0, u8_range, out_f32, out_u8, range_acc, num_sms, s); break;
        }
        if (e != cudaSuccess) return e;
        return cudaSuccess;
    }
    long long n = P - p_tail;
    long long grid = (n + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    k_project_s<F32, U8, RNG><<<static_cast<unsigned>(grid), TPB, 0, s>>>(cube, B, P, p_tail, dm, j0, kc, u8_range,
                                                                     out_f32, out_u8, range_acc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_range_init(float* range, int k, cudaStream_t s)
{
    k_range_init<<<1, 64, 0, s>>>(range, k);
    return cudaGetLastError();
}

cudaError_t launch_train_range(int B, int K, const uint16_t* xtr, DevModel* dm, int nvec, int num_sms,
                               cudaStream_t s)
{
    const unsigned grid = static_cast<unsigned>(num_sms) * 4;
    for (int j0 = 0; j0 < nvec; j0 += KCH) {
        const int kc = (nvec - j0) < KCH ? (nvec - j0) : KCH;
        switch (kc) {
            case 1: k_train_range<1><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 2: k_train_range<2><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 3: k_train_range<3><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 4: k_train_range<4><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 5: k_train_range<5><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 6: k_train_range<6><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            case 7: k_train_range<7><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
            default: k_train_range<8><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0); break;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_batch_train_range(const PageDev* pages, int n, const BatchTotals* tot,
                                     const uint16_t* xtr_pool, int max_k, int num_sms, cudaStream_t s)
{
    const int grid = num_sms * 4;
    switch (max_k) {
        case 1: kb_train_range<1><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 2: kb_train_range<2><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 3: kb_train_range<3><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 4: kb_train_range<4><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 5: kb_train_range<5><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 6: kb_train_range<6><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 7: kb_train_range<7><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        case 8: kb_train_range<8><<<grid, TPB, 0, s>>>(pages, n, tot, xtr_pool); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_project(const PageDev* pages, const int* item_page, long long it_begin, long long it_end,
                                 int groups_per_item, int grid, int k, cudaStream_t s)
{
    const long long items = it_end - it_begin;
    if (items < 1) return cudaSuccess;
    const long long g = grid < items ? grid : items;
    const int contiguous = g < items ? 1 : 0;
    const unsigned gx = static_cast<unsigned>(g);
    switch (k) {
        case 1: kb_project_v8<1><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 2: kb_project_v8<2><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 3: kb_project_v8<3><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 4: kb_project_v8<4><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 5: kb_project_v8<5><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 6: kb_project_v8<6><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 7: kb_project_v8<7><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        case 8: kb_project_v8<8><<<gx, TPB, 0, s>>>(pages, item_page, it_begin, it_end, groups_per_item, contiguous); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_project(const uint16_t* cube, int B, long long P, const DevModel* dm, int k,
                           float* out_f32, uint8_t* out_u8, const float* u8_range, float* range_acc,
                           int num_sms, cudaStream_t s)
{
    const bool aligned = (P % 8 == 0) && (reinterpret_cast<uintptr_t>(cube) % 16 == 0) &&
                         (!out_f32 || reinterpret_cast<uintptr_t>(out_f32) % 16 == 0) &&
                         (!out_u8 || reinterpret_cast<uintptr_t>(out_u8) % 8 == 0);
    const bool f32 = out_f32 != nullptr, u8 = out_u8 != nullptr, rng = range_acc != nullptr;
    for (int j0 = 0; j0 < k; j0 += KCH) {
        const int kc = (k - j0) < KCH ? (k - j0) : KCH;
        cudaError_t e;
        if (f32 && !u8 && !rng)
            e = run_chunk<true, false, false>(cube, B, P, dm, j0, kc, u8_range, out_f32, out_u8, range_acc, aligned, num_sms, s);
        else if (f32 && !u8 && rng)
            e = run_chunk<true, false, true>(cube, B, P, dm, j0, kc, u8_range, out_f32, out_u8, range_acc, aligned, num_sms, s);
        else if (!f32 && !u8 && rng)
            e = run_chunk<false, false, true>(cube, B, P, dm, j0, kc, u8_range, out_f32, out_u8, range_acc, aligned, num_sms, s);
        else if (!f32 && u8 && !rng)
            e = run_chunk<false, true, false>(cube, B, P, dm, j0, kc, u8_range, out_f32, out_u8, range_acc, aligned, num_sms, s);
        else
            return cudaErrorInvalidValue;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_f32_range(const float* proj, int k, long long P, const DevModel*, float* range_acc,
                             int num_sms, cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(proj) % 16 == 0 && P % 4 == 0) ? 1 : 0;
    long long gx = (P / 4 + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    k_f32_range<<<dim3(static_cast<unsigned>(gx), k), TPB, 0, s>>>(proj, k, P, vec, range_acc);
    return cudaGetLastError();
}

cudaError_t launch_f32_to_u8(const float* proj, int k, long long P, const DevModel*, const float* range,
                             uint8_t* out, int num_sms, cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(proj) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 4 == 0 &&
                     P % 4 == 0) ? 1 : 0;
    long long gx = (P / 4 + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    k_f32_to_u8<<<dim3(static_cast<unsigned>(gx), k), TPB, 0, s>>>(proj, k, P, vec, range, out);
    return cudaGetLastError();
}

}  // namespace cva
