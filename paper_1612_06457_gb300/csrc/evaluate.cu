// evaluate.cu -- the paper's evaluation and presentation of the enhanced
// images, on the device.
//
// Cluster-separation indices (Section 3, eqs. 1-5, p = 2) of the labelled
// classes in a k-band image (the 8-bit images, or the FP32 projections):
// class centroids A_c, scatters S_c (mean Euclidean distance to the
// centroid), centroid distances M_ij, Davies-Bouldin ratios
// R_ij = (S_i + S_j) / M_ij and Dunn indices DI_ij = (M_ij - S_i - S_j) /
// max(S_i, S_j).  Two passes over the labelled pixels (sums, then
// distances), each a per-CTA shared-memory reduction merged with atomics,
// then one CTA for the K x K tables.  8-bit sums are exact 64-bit integers;
// distances accumulate in FP64.
//
// RGB composite (Section 2 / Figure 5: three grayscale images as the red,
// green and blue channels, the one with the clearest undertext in green;
// optionally inverted): one HBM pass, 3 bytes in and 3 out per pixel.
#include <math.h>

#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;

template <bool F32>
__device__ inline double pixel_value(const uint8_t* u8, const float* f32, long long i)
{
    return F32 ? static_cast<double>(f32[i]) : static_cast<double>(u8[i]);
}

__global__ void k_ev_reset(DevModel* __restrict__ dm, int k, int K)
{
    for (int i = threadIdx.x; i < MAXK * MAXB; i += blockDim.x) dm->ev_sum[i / MAXB][i % MAXB] = 0.0;
    if (threadIdx.x < MAXK) {
        dm->ev_count[threadIdx.x] = 0ull;
        dm->ev_scatter[threadIdx.x] = 0.0;
    }
    if (threadIdx.x == 0) dm->ev_status = CVA_OK;
}

// Pass 1: per-class counts and sums of the labelled pixels.
template <bool F32>
__global__ void __launch_bounds__(TPB)
k_ev_sums(const uint8_t* __restrict__ u8, const float* __restrict__ f32, int k, long long P,
          const uint8_t* __restrict__ labels, int K, DevModel* __restrict__ dm)
{
    __shared__ unsigned long long cnt[MAXK];
    __shared__ double sum[MAXK][MAXB];
    __shared__ int bad;
    for (int i = threadIdx.x; i < MAXK * MAXB; i += TPB) sum[i / MAXB][i % MAXB] = 0.0;
    if (threadIdx.x < MAXK) cnt[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    for (long long p = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x; p < P; p += stride) {
        const int lab = labels[p];
        if (lab == 0) continue;
        if (lab > K) {
            bad = 1;
            continue;
        }
        atomicAdd(&cnt[lab - 1], 1ull);
        for (int j = 0; j < k; ++j) atomicAdd(&sum[lab - 1][j], pixel_value<F32>(u8, f32, static_cast<long long>(j) * P + p));
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad) atomicCAS(&dm->ev_status, 0, CVA_ERR_LABEL_RANGE);
    for (int i = threadIdx.x; i < K * k; i += TPB) {
        const int c = i / k, j = i - (i / k) * k;
        if (sum[c][j] != 0.0) atomicAdd(&dm->ev_sum[c][j], sum[c][j]);
    }
    if (threadIdx.x < K && cnt[threadIdx.x]) atomicAdd(&dm->ev_count[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void k_ev_centroids(DevModel* __restrict__ dm, int k, int K)
{
    for (int i = threadIdx.x; i < K * k; i += blockDim.x) {
        const int c = i / k, j = i - (i / k) * k;
        const unsigned long long n = dm->ev_count[c];
        dm->ev_sum[c][j] = n ? dm->ev_sum[c][j] / static_cast<double>(n) : 0.0;
    }
    if (threadIdx.x < K && dm->ev_count[threadIdx.x] == 0ull) atomicCAS(&dm->ev_status, 0, CVA_ERR_EMPTY_CLASS);
}

// Pass 2: per-class sums of the pixels' distances to their centroid.
template <bool F32>
__global__ void __launch_bounds__(TPB)
k_ev_scatter(const uint8_t* __restrict__ u8, const float* __restrict__ f32, int k, long long P,
             const uint8_t* __restrict__ labels, int K, DevModel* __restrict__ dm)
{
    __shared__ double cen[MAXK][MAXB];
    __shared__ double dsum[MAXK];
    for (int i = threadIdx.x; i < K * k; i += TPB) cen[i / k][i % k] = dm->ev_sum[i / k][i % k];
    if (threadIdx.x < MAXK) dsum[threadIdx.x] = 0.0;
    __syncthreads();
    if (dm->ev_status != 0) return;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    for (long long p = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x; p < P; p += stride) {
        const int lab = labels[p];
        if (lab == 0 || lab > K) continue;
        double d2 = 0.0;
        for (int j = 0; j < k; ++j) {
            const double d = pixel_value<F32>(u8, f32, static_cast<long long>(j) * P + p) - cen[lab - 1][j];
            d2 = fma(d, d, d2);
        }
        atomicAdd(&dsum[lab - 1], sqrt(d2));
    }
    __syncthreads();
    if (threadIdx.x < K && dsum[threadIdx.x] != 0.0) atomicAdd(&dm->ev_scatter[threadIdx.x], dsum[threadIdx.x]);
}

// The K x K tables (eqs. 2, 3 and 5).
__global__ void k_ev_tables(DevModel* __restrict__ dm, int k, int K)
{
    __shared__ double S[MAXK];
    if (dm->ev_status != 0) return;
    if (threadIdx.x < K) S[threadIdx.x] = dm->ev_scatter[threadIdx.x] / static_cast<double>(dm->ev_count[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x < K) dm->ev_scatter[threadIdx.x] = S[threadIdx.x];
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
        const int a = i / K, b = i - (i / K) * K;
        double d2 = 0.0;
        for (int j = 0; j < k; ++j) {
            const double d = dm->ev_sum[a][j] - dm->ev_sum[b][j];
            d2 = fma(d, d, d2);
        }
        const double m = sqrt(d2);
        dm->ev_M[a][b] = m;
        if (a == b) {
            dm->ev_R[a][b] = 0.0;
            dm->ev_DI[a][b] = 0.0;
        } else {
            const double inf = __longlong_as_double(0x7FF0000000000000ll);
            const double smax = fmax(S[a], S[b]);
            dm->ev_R[a][b] = m > 0.0 ? (S[a] + S[b]) / m : inf;
            dm->ev_DI[a][b] = smax > 0.0 ? (m - S[a] - S[b]) / smax : inf;
        }
    }
}

__global__ void __launch_bounds__(TPB)
k_rgb(const uint8_t* __restrict__ planes, long long P, int s0, int s1, int s2, int invert, int vec,
      uint8_t* __restrict__ rgb)
{
    const uint8_t* r = planes + static_cast<long long>(s0) * P;
    const uint8_t* g = planes + static_cast<long long>(s1) * P;
    const uint8_t* b = planes + static_cast<long long>(s2) * P;
    const uint32_t xr = (invert & 1) ? 0xFFFFFFFFu : 0u, xg = (invert & 2) ? 0xFFFFFFFFu : 0u,
                   xb = (invert & 4) ? 0xFFFFFFFFu : 0u;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    const long long start = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x;
    long long done = 0;
    if (vec) {  // 4 pixels a step: three 4-byte loads, three 4-byte stores
        const long long n4 = P / 4;
        for (long long q = start; q < n4; q += stride) {
            const uint32_t vr = __ldcs(reinterpret_cast<const unsigned int*>(r) + q) ^ xr;
            const uint32_t vg = __ldcs(reinterpret_cast<const unsigned int*>(g) + q) ^ xg;
            const uint32_t vb = __ldcs(reinterpret_cast<const unsigned int*>(b) + q) ^ xb;
            // r0 g0 b0 r1 | g1 b1 r2 g2 | b2 r3 g3 b3
            const uint32_t w0 = (vr & 0xFFu) | ((vg & 0xFFu) << 8) | ((vb & 0xFFu) << 16) | ((vr & 0xFF00u) << 16);
            const uint32_t w1 = ((vg >> 8) & 0xFFu) | (((vb >> 8) & 0xFFu) << 8) | (((vr >> 16) & 0xFFu) << 16) |
                                (((vg >> 16) & 0xFFu) << 24);
            const uint32_t w2 = ((vb >> 16) & 0xFFu) | (((vr >> 24) & 0xFFu) << 8) | (((vg >> 24) & 0xFFu) << 16) |
                                (((vb >> 24) & 0xFFu) << 24);
            unsigned int* dst = reinterpret_cast<unsigned int*>(rgb) + 3 * q;
            __stcs(dst, w0);
            __stcs(dst + 1, w1);
            __stcs(dst + 2, w2);
        }
        done = n4 * 4;
    }
    for (long long p = done + start; p < P; p += stride) {
        rgb[3 * p] = static_cast<uint8_t>(r[p] ^ (xr & 0xFFu));
        rgb[3 * p + 1] = static_cast<uint8_t>(g[p] ^ (xg & 0xFFu));
        rgb[3 * p + 2] = static_cast<uint8_t>(b[p] ^ (xb & 0xFFu));
    }
}

int grid_for(long long units, int num_sms, int per_sm)
{
    long long g = (units + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * per_sm;
    if (g > cap) g = cap;
    return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_cluster_indices(const uint8_t* img_u8, const float* img_f32, int k, long long P,
                                   const uint8_t* labels, int K, DevModel* dm, int num_sms, cudaStream_t s)
{
    const int grid = grid_for(P, num_sms, 4);
    k_ev_reset<<<1, 256, 0, s>>>(dm, k, K);
    if (img_f32) k_ev_sums<true><<<grid, TPB, 0, s>>>(img_u8, img_f32, k, P, labels, K, dm);
    else k_ev_sums<false><<<grid, TPB, 0, s>>>(img_u8, img_f32, k, P, labels, K, dm);
    k_ev_centroids<<<1, 256, 0, s>>>(dm, k, K);
    if (img_f32) k_ev_scatter<true><<<grid, TPB, 0, s>>>(img_u8, img_f32, k, P, labels, K, dm);
    else k_ev_scatter<false><<<grid, TPB, 0, s>>>(img_u8, img_f32, k, P, labels, K, dm);
    k_ev_tables<<<1, 256, 0, s>>>(dm, k, K);
    return cudaGetLastError();
}

cudaError_t launch_rgb_composite(const uint8_t* planes, long long P, int s0, int s1, int s2, int invert,
                                 uint8_t* rgb, int num_sms, cudaStream_t s)
{
    const int vec = (P % 4 == 0) && (reinterpret_cast<uintptr_t>(planes) % 4 == 0) &&
                    (reinterpret_cast<uintptr_t>(rgb) % 4 == 0);
    k_rgb<<<grid_for(P / 4 + 1, num_sms, 8), TPB, 0, s>>>(planes, P, s0, s1, s2, invert, vec, rgb);
    return cudaGetLastError();
}

}  // namespace cva
