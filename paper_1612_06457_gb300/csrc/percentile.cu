// percentile.cu -- the third rescale's range: the projections with p percent
// of the pixels taken out of each tail (Section 2 takes out the 0.01, 0.1, 1
// or 5 percentiles of the projected data before the same linear rescale).
//
// With m = floor(p P / 100) values taken out at each end, lo_j is the
// (m+1)-th smallest and hi_j the (m+1)-th largest of the P float32 values of
// projection j.  Both are exact order statistics, found by a radix select on
// the order-preserving 32-bit keys of the floats in three passes of 11, 11
// and 10 bits: each pass histograms, per variate and per target (lo, hi), the
// next digit of the keys that match the target's known prefix, then one CTA
// per variate finds the bin holding the target's rank and extends the prefix.
// Every pass reads the projections once (HBM-bound); the histograms are
// privatized in shared memory (per warp in the first pass, where every key
// counts and many share the leading digits).
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int NBIN = 2048;

__device__ inline uint32_t float_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ inline float key_float(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Digit of pass s and the mask of the bits fixed before it.
template <int S>
__device__ inline uint32_t digit(uint32_t key)
{
    return S == 0 ? (key >> 21) : S == 1 ? ((key >> 10) & 0x7FFu) : (key & 0x3FFu);
}

template <int S>
__host__ __device__ constexpr uint32_t prefix_mask()
{
    return S == 0 ? 0u : S == 1 ? 0xFFE00000u : 0xFFFFFC00u;
}

__global__ void k_sel_init(DevModel* __restrict__ dm, int k, unsigned int m, unsigned int P)
{
    const int i = threadIdx.x;
    if (i < 2 * k) {
        dm->sel_prefix[i] = 0u;
        dm->sel_rank[i] = (i & 1) ? (P - 1u - m) : m;  // 0-based ranks of lo and hi
    }
}

// Passes 1 and 2: only keys that match a target's prefix are counted (few),
// into that target's shared histogram.
template <int S>
__device__ inline void count_key(uint32_t key, uint32_t p_lo, uint32_t p_hi, unsigned int* h)
{
    const uint32_t d = digit<S>(key);
    if ((key & prefix_mask<S>()) == p_lo) atomicAdd(h + d, 1u);
    if ((key & prefix_mask<S>()) == p_hi) atomicAdd(h + NBIN + d, 1u);
}

// Pass S: histograms of the next digit for both targets of variate
// blockIdx.y, merged into hist[j][t][bin].  In pass 0 every key counts for
// both targets, so one histogram serves both (row t = 0), kept per warp in
// shared memory to spread the atomics of keys with equal leading digits.
template <int S>
__global__ void __launch_bounds__(TPB)
k_sel_hist(const float* __restrict__ proj, long long P, int vec, const DevModel* __restrict__ dm,
           unsigned int* __restrict__ hist)
{
    extern __shared__ unsigned int hs[];  // S == 0: NWARP x NBIN; else 2 x NBIN
    constexpr int NWARP = TPB / 32;
    constexpr int NH = S == 0 ? NWARP : 2;
    const int j = blockIdx.y, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NH * NBIN; i += TPB) hs[i] = 0u;
    const uint32_t p_lo = dm->sel_prefix[2 * j], p_hi = dm->sel_prefix[2 * j + 1];
    __syncthreads();
    unsigned int* hw = hs + warp * NBIN;
    const float* src = proj + static_cast<long long>(j) * P;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    const long long start = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = P / 4;
        for (long long g = start; g < n4; g += stride) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(src) + g);
            if (S == 0) {
                atomicAdd(hw + digit<0>(float_key(v.x)), 1u);
                atomicAdd(hw + digit<0>(float_key(v.y)), 1u);
                atomicAdd(hw + digit<0>(float_key(v.z)), 1u);
                atomicAdd(hw + digit<0>(float_key(v.w)), 1u);
            } else {
                count_key<S>(float_key(v.x), p_lo, p_hi, hs);
                count_key<S>(float_key(v.y), p_lo, p_hi, hs);
                count_key<S>(float_key(v.z), p_lo, p_hi, hs);
                count_key<S>(float_key(v.w), p_lo, p_hi, hs);
            }
        }
        done = n4 * 4;
    }
    for (long long p = done + start; p < P; p += stride) {
        const uint32_t key = float_key(src[p]);
        if (S == 0) atomicAdd(hw + digit<0>(key), 1u);
        else count_key<S>(key, p_lo, p_hi, hs);
    }
    __syncthreads();
    unsigned int* g = hist + static_cast<long long>(j) * 2 * NBIN;
    if (S == 0) {
        for (int i = threadIdx.x; i < NBIN; i += TPB) {
            unsigned int c = 0;
            #pragma unroll
            for (int w = 0; w < NWARP; ++w) c += hs[w * NBIN + i];
            if (c) atomicAdd(g + i, c);
        }
    } else {
        for (int i = threadIdx.x; i < 2 * NBIN; i += TPB) {
            const unsigned int c = hs[i];
            if (c) atomicAdd(g + i, c);
        }
    }
}

// One CTA per variate: the bin of each target's rank, the extended prefix and
// the rank within the bin; the histograms are cleared for the next pass.  The
// last pass writes the range.
template <int S>
__global__ void __launch_bounds__(TPB)
k_sel_pick(DevModel* __restrict__ dm, unsigned int* __restrict__ hist, float* __restrict__ range_out)
{
    constexpr int PER = NBIN / TPB;  // 8 bins a thread
    __shared__ unsigned int wsum[TPB / 32];
    __shared__ unsigned int s_bin, s_before;
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned int* g = hist + static_cast<long long>(j) * 2 * NBIN;
    for (int t = 0; t < 2; ++t) {
        const unsigned int rank = dm->sel_rank[2 * j + t];
        if (tid == 0) {
            s_bin = 0u;
            s_before = 0u;
        }
        const int row = S == 0 ? 0 : t;  // pass 0 keeps one histogram for both targets
        unsigned int c[PER], sum = 0;
        #pragma unroll
        for (int i = 0; i < PER; ++i) {
            c[i] = g[row * NBIN + tid * PER + i];
            sum += c[i];
        }
        unsigned int v = sum;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        unsigned int before = v - sum;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        if (rank >= before && rank < before + sum) {
            unsigned int run = before;
            #pragma unroll
            for (int i = 0; i < PER; ++i) {
                if (rank >= run && rank < run + c[i]) {
                    s_bin = static_cast<unsigned int>(tid * PER + i);
                    s_before = run;
                }
                run += c[i];
            }
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t shift = S == 0 ? 21u : S == 1 ? 10u : 0u;
            const uint32_t prefix = dm->sel_prefix[2 * j + t] | (s_bin << shift);
            dm->sel_prefix[2 * j + t] = prefix;
            dm->sel_rank[2 * j + t] = rank - s_before;
            if (S == 2) range_out[2 * j + t] = key_float(prefix);
        }
        __syncthreads();
    }
    for (int i = tid; i < 2 * NBIN; i += TPB) g[i] = 0u;
}

}  // namespace

cudaError_t launch_percentile_range(const float* proj, int k, long long P, long long m, DevModel* dm,
                                    unsigned int* hist, float* range_out, int num_sms, cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(proj) % 16 == 0 && P % 4 == 0) ? 1 : 0;
    long long gx = (P / 4 + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 4;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(k));
    const int smem0 = (TPB / 32) * NBIN * static_cast<int>(sizeof(unsigned int));
    const int smem1 = 2 * NBIN * static_cast<int>(sizeof(unsigned int));
    cudaError_t e = cudaFuncSetAttribute(k_sel_hist<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem0);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 2 * NBIN * k, s);
    if (e != cudaSuccess) return e;
    k_sel_init<<<1, 2 * MAXB, 0, s>>>(dm, k, static_cast<unsigned int>(m), static_cast<unsigned int>(P));
    k_sel_hist<0><<<grid, TPB, smem0, s>>>(proj, P, vec, dm, hist);
    k_sel_pick<0><<<k, TPB, 0, s>>>(dm, hist, range_out);
    k_sel_hist<1><<<grid, TPB, smem1, s>>>(proj, P, vec, dm, hist);
    k_sel_pick<1><<<k, TPB, 0, s>>>(dm, hist, range_out);
    k_sel_hist<2><<<grid, TPB, smem1, s>>>(proj, P, vec, dm, hist);
    k_sel_pick<2><<<k, TPB, 0, s>>>(dm, hist, range_out);
    return cudaGetLastError();
}

}  // namespace cva
