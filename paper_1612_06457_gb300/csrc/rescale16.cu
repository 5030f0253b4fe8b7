// rescale16.cu -- the 16-bit image of the linear rescale (Section 2's CVA-GSL
// tool writes 8- and 16-bit images): out = floor(65535 (y - lo) / (hi - lo)
// + 1/2) clamped to 0..65535, 0 when hi <= lo.  One pass over the float32
// projections (4 bytes in, 2 out per pixel), bound by HBM bandwidth.
#include "cva_internal.cuh"

namespace cva {

namespace {

constexpr int TPB = 256;

__device__ inline float scale16(float lo, float hi)
{
    const float w = __fsub_rn(hi, lo);
    return (w > 0.0f && w < 3.0e38f) ? __fdiv_rn(65535.0f, w) : 0.0f;
}

// (y - lo) is formed first, so the scale multiplies a small difference.
__device__ inline uint32_t code16(float y, float lo, float sc)
{
    const float t = fminf(fmaxf(__fmaf_rn(__fsub_rn(y, lo), sc, 0.5f), 0.0f), 65535.0f);
    return static_cast<uint32_t>(__float2int_rd(t));
}

__global__ void __launch_bounds__(TPB)
k_f32_to_u16(const float* __restrict__ proj, long long P, int vec, const float* __restrict__ range,
             uint16_t* __restrict__ out)
{
    const int j = blockIdx.y;
    const float lo = range[2 * j];
    const float sc = scale16(lo, range[2 * j + 1]);
    const float* src = proj + static_cast<long long>(j) * P;
    uint16_t* dst = out + static_cast<long long>(j) * P;
    const long long stride = static_cast<long long>(gridDim.x) * TPB;
    const long long start = static_cast<long long>(blockIdx.x) * TPB + threadIdx.x;
    long long done = 0;
    if (vec) {
        const long long n4 = P / 4;
        for (long long g = start; g < n4; g += stride) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(src) + g);
            const uint2 c = make_uint2(code16(v.x, lo, sc) | (code16(v.y, lo, sc) << 16),
                                       code16(v.z, lo, sc) | (code16(v.w, lo, sc) << 16));
            __stcs(reinterpret_cast<uint2*>(dst) + g, c);
        }
        done = n4 * 4;
    }
    for (long long p = done + start; p < P; p += stride) dst[p] = static_cast<uint16_t>(code16(src[p], lo, sc));
}

}  // namespace

cudaError_t launch_f32_to_u16(const float* proj, int k, long long P, const float* range, uint16_t* out,
                              int num_sms, cudaStream_t s)
{
    const int vec = (reinterpret_cast<uintptr_t>(proj) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 8 == 0 &&
                     P % 4 == 0) ? 1 : 0;
    long long gx = (P / 4 + TPB - 1) / TPB;
    const long long cap = static_cast<long long>(num_sms) * 8;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    k_f32_to_u16<<<dim3(static_cast<unsigned>(gx), k), TPB, 0, s>>>(proj, P, vec, range, out);
    return cudaGetLastError();
}

}  // namespace cva
