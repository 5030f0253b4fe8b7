// project64.cu -- the FP64 form of the projection and of the training range
// (CVA_PRECISION_FP64).
//
// The same quantities as project.cu (Section 2: the canonical coefficients
// multiplied with the band images, each result mapped onto 0..255 by its own
// range over all pixels or by the training points' range), with FP64
// coefficients, FP64 centring and FP64 accumulation:
//     y_j[p] = sum_b V[b][j] (x_b[p] - mu_b)
//     code   = floor((y - lo) * (255 / (hi - lo)) + 1/2), clamped to 0..255.
// It is the plain high-precision form that the FP32 path is measured
// against: FP64 issues at a small fraction of the FP32 rate on this part, so
// this pass is bound by the FP64 pipe (B k fused multiply-adds per pixel),
// not by HBM.  One pixel per thread in a grid-stride loop; the coefficients
// sit in shared memory and are read as broadcasts.
//
// Ranges are kept as (min, max) pairs of order-preserving 64-bit encodings
// (ord_enc_bits), reduced per warp and merged with integer atomics.
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;
constexpr int KCH = 8;  // variates per pass

struct Coef64 {
    double V[MAXB][KCH];
    double mu[MAXB];
    double lo[KCH];
    double scale[KCH];
};

__device__ inline unsigned long long enc(double d)
{
    return ord_enc_bits(static_cast<unsigned long long>(__double_as_longlong(d)));
}

__device__ inline double dec(unsigned long long u)
{
    return __longlong_as_double(static_cast<long long>(ord_dec_bits(u)));
}

// 255 / (hi - lo), or 0 when the range is empty (every code is then 0).
__device__ inline double scale64(double lo, double hi)
{
    return hi > lo ? 255.0 / (hi - lo) : 0.0;
}

__device__ inline uint8_t code64(double y, double lo, double scale)
{
    double t = floor(fma(y - lo, scale, 0.5));
    t = fmin(fmax(t, 0.0), 255.0);
    return static_cast<uint8_t>(static_cast<int>(t));
}

__device__ void load_coef64(Coef64& c, const DevModel* dm, int B, int j0, int kc,
                            const unsigned long long* u8_enc, const float* u8_range)
{
    for (int e = threadIdx.x; e < MAXB * KCH; e += TPB) {
        const int b = e / KCH, j = e % KCH;
        c.V[b][j] = (b < B && j < kc) ? dm->V[b][j0 + j] : 0.0;
    }
    if (threadIdx.x < MAXB) c.mu[threadIdx.x] = threadIdx.x < B ? dm->mu[threadIdx.x] : 0.0;
    if (threadIdx.x < KCH) {
        const int j = threadIdx.x;
        double lo = 0.0, hi = 0.0;
        if (j < kc && u8_enc) {
            lo = dec(u8_enc[2 * (j0 + j)]);
            hi = dec(u8_enc[2 * (j0 + j) + 1]);
        } else if (j < kc && u8_range) {
            lo = static_cast<double>(u8_range[2 * (j0 + j)]);
            hi = static_cast<double>(u8_range[2 * (j0 + j) + 1]);
        }
        c.lo[j] = lo;
        c.scale[j] = scale64(lo, hi);
    }
}

// Per-warp reduction of KC (min, max) pairs, then one atomic pair per warp.
template <int KC>
__device__ inline void merge_range(double (&mn)[KC], double (&mx)[KC], unsigned long long* acc, int j0, int kc)
{
    #pragma unroll
    for (int j = 0; j < KC; ++j) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[j] = fmin(mn[j], __shfl_xor_sync(0xFFFFFFFFu, mn[j], o));
            mx[j] = fmax(mx[j], __shfl_xor_sync(0xFFFFFFFFu, mx[j], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        #pragma unroll
        for (int j = 0; j < KC; ++j) {
            if (j < kc && mn[j] <= mx[j]) {
                atomicMin(acc + 2 * (j0 + j), enc(mn[j]));
                atomicMax(acc + 2 * (j0 + j) + 1, enc(mx[j]));
            }
        }
    }
}

template <int KV, bool F32, bool U8, bool RNG>
__global__ void __launch_bounds__(TPB)
k_project64(const uint16_t* __restrict__ cube, int B, long long P, const DevModel* __restrict__ dm, int j0, int kc,
            float* __restrict__ out_f32, uint8_t* __restrict__ out_u8, const unsigned long long* u8_enc,
            const float* u8_range, unsigned long long* enc_acc)
{
    __shared__ Coef64 c;
    if (dm->status != 0 || !dm->fitted) return;
    load_coef64(c, dm, B, j0, kc, U8 ? u8_enc : nullptr, U8 ? u8_range : nullptr);
    __syncthreads();
    double mn[KV], mx[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) { mn[j] = __longlong_as_double(0x7FF0000000000000ll); mx[j] = -mn[j]; }
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    for (long long p = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x; p < P; p += stride) {
        double acc[KV];
        #pragma unroll
        for (int j = 0; j < KV; ++j) acc[j] = 0.0;
        for (int b = 0; b < B; ++b) {
            const double xs = static_cast<double>(__ldg(cube + static_cast<long long>(b) * P + p)) - c.mu[b];
            #pragma unroll
            for (int j = 0; j < KV; ++j) acc[j] = fma(c.V[b][j], xs, acc[j]);
        }
        #pragma unroll
        for (int j = 0; j < KV; ++j) {
            if (j < kc) {
                const long long o = static_cast<long long>(j0 + j) * P + p;
                if (F32) __stcs(out_f32 + o, static_cast<float>(acc[j]));
                if (U8) out_u8[o] = code64(acc[j], c.lo[j], c.scale[j]);
                if (RNG) { mn[j] = fmin(mn[j], acc[j]); mx[j] = fmax(mx[j], acc[j]); }
            }
        }
    }
    if (RNG) merge_range<KV>(mn, mx, enc_acc, j0, kc);
}

// FP64 scores of the training pixels (rows of the gathered training matrix:
// x_0 .. x_{B-1}, 1, 0 ..) and their extremes.
template <int KV>
__global__ void __launch_bounds__(TPB)
k_train_range64(int B, int K, const uint16_t* __restrict__ xtr, DevModel* __restrict__ dm, int j0, int kc)
{
    __shared__ Coef64 c;
    if (dm->status != 0 || !dm->fitted) return;
    load_coef64(c, dm, B, j0, kc, nullptr, nullptr);
    __syncthreads();
    unsigned int N = 0;
    for (int cl = 0; cl < K; ++cl) N += dm->cls_count[cl];
    const int BR = xtr_row(B);
    double mn[KV], mx[KV];
    #pragma unroll
    for (int j = 0; j < KV; ++j) { mn[j] = __longlong_as_double(0x7FF0000000000000ll); mx[j] = -mn[j]; }
    const unsigned int stride = gridDim.x * TPB;
    for (unsigned int i = blockIdx.x * TPB + threadIdx.x; i < N; i += stride) {
        const uint16_t* row = xtr + static_cast<long long>(i) * BR;
        double acc[KV];
        #pragma unroll
        for (int j = 0; j < KV; ++j) acc[j] = 0.0;
        for (int b = 0; b < B; ++b) {
            const double xs = static_cast<double>(__ldg(row + b)) - c.mu[b];
            #pragma unroll
            for (int j = 0; j < KV; ++j) acc[j] = fma(c.V[b][j], xs, acc[j]);
        }
        #pragma unroll
        for (int j = 0; j < KV; ++j) { mn[j] = fmin(mn[j], acc[j]); mx[j] = fmax(mx[j], acc[j]); }
    }
    merge_range<KV>(mn, mx, dm->train_enc64, j0, kc);
}

__global__ void k_enc_init(unsigned long long* enc, int k)
{
    const int i = threadIdx.x;
    if (i < 2 * k) enc[i] = (i & 1) ? 0ull : ~0ull;
}

__global__ void k_enc_to_float(const unsigned long long* enc, int k, float* out)
{
    const int i = threadIdx.x;
    if (i < 2 * k) out[i] = static_cast<float>(dec(enc[i]));
}

int grid_for(long long units, int num_sms)
{
    const long long want = (units + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 8;
    return static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
}

}  // namespace

cudaError_t launch_enc_init(unsigned long long* enc, int k, cudaStream_t s)
{
    k_enc_init<<<1, 2 * MAXB, 0, s>>>(enc, k);
    return cudaGetLastError();
}

cudaError_t launch_enc_to_float(const unsigned long long* enc, int k, float* out, cudaStream_t s)
{
    k_enc_to_float<<<1, 2 * MAXB, 0, s>>>(enc, k, out);
    return cudaGetLastError();
}

cudaError_t launch_train_range64(int B, int K, const uint16_t* xtr, DevModel* dm, int nvec, int num_sms,
                                 cudaStream_t s)
{
    cudaError_t e = launch_enc_init(dm->train_enc64, nvec, s);
    const int grid = num_sms * 2;
    for (int j0 = 0; j0 < nvec && e == cudaSuccess; j0 += KCH) {
        const int kc = (nvec - j0) < KCH ? (nvec - j0) : KCH;
        switch (kc) {
            case 1: k_train_range64<1><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 2: k_train_range64<2><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 3: k_train_range64<3><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 4: k_train_range64<4><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 5: k_train_range64<5><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 6: k_train_range64<6><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            case 7: k_train_range64<7><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
            default: k_train_range64<8><<<grid, TPB, 0, s>>>(B, K, xtr, dm, j0, kc); break;
        }
        e = cudaGetLastError();
    }
    return e;
}

template <int KV>
cudaError_t run64(const uint16_t* cube, int B, long long P, const DevModel* dm, int j0, int kc, float* out_f32,
                  uint8_t* out_u8, const unsigned long long* u8_enc, const float* u8_range,
                  unsigned long long* enc_acc, int grid, cudaStream_t s)
{
    const bool f32 = out_f32 != nullptr, u8 = out_u8 != nullptr, rng = enc_acc != nullptr;
    if (f32 && !u8 && !rng)
        k_project64<KV, true, false, false><<<grid, TPB, 0, s>>>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc);
    else if (f32 && !u8 && rng)
        k_project64<KV, true, false, true><<<grid, TPB, 0, s>>>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc);
    else if (!f32 && !u8 && rng)
        k_project64<KV, false, false, true><<<grid, TPB, 0, s>>>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc);
    else if (!f32 && u8 && !rng)
        k_project64<KV, false, true, false><<<grid, TPB, 0, s>>>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc);
    else if (f32 && u8 && !rng)
        k_project64<KV, true, true, false><<<grid, TPB, 0, s>>>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_project64(const uint16_t* cube, int B, long long P, const DevModel* dm, int k,
                             float* out_f32, uint8_t* out_u8, const unsigned long long* u8_enc,
                             const float* u8_range, unsigned long long* enc_acc, int num_sms, cudaStream_t s)
{
    const int grid = grid_for(P, num_sms);
    for (int j0 = 0; j0 < k; j0 += KCH) {
        const int kc = (k - j0) < KCH ? (k - j0) : KCH;
        cudaError_t e;
        switch (kc) {
            case 1: e = run64<1>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 2: e = run64<2>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 3: e = run64<3>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 4: e = run64<4>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 5: e = run64<5>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 6: e = run64<6>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            case 7: e = run64<7>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
            default: e = run64<8>(cube, B, P, dm, j0, kc, out_f32, out_u8, u8_enc, u8_range, enc_acc, grid, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cva
