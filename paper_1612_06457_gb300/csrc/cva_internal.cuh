// cva_internal.cuh -- device model layout, launch helpers and small device
// utilities shared by the CUDA translation units of the CVA library.
//
// Nothing here is part of the C ABI (include/cva.h); the model block below
// lives in device memory and is owned by a cva_model.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cva.h"

namespace cva {

constexpr int MAXB = CVA_MAX_BANDS;                     // 32 bands
constexpr int MAXK = CVA_MAX_CLASSES;                   // 16 classes
constexpr int MAXBA = ((MAXB + 1 + 3) / 4) * 4;         // augmented bands, padded to 4: 36
constexpr int MAXNB = MAXBA / 4;                        // 4-band blocks: 9
constexpr int MAXBLK = MAXNB * (MAXNB + 1) / 2;         // upper-triangle block pairs: 45
constexpr int LABEL_TILE = 16384;                       // labels per CTA of the label passes
constexpr long long MAX_PIXELS = 1LL << 31;             // H W limit of the ABI
constexpr int MAX_TILES = static_cast<int>(MAX_PIXELS / LABEL_TILE);  // 131072

// Pivot test of the Cholesky factorization: Sw is "not positive definite"
// when a pivot is not above this multiple of its own diagonal entry.
constexpr double PIVOT_REL = 1e-12;
// Eigenvector sign convention: components within this relative distance of
// the largest magnitude tie, and the lowest band index wins.
constexpr double TIE_REL = 1e-12;
// 2^23 as a float: or-ing a 16-bit integer into its mantissa gives 2^23 + x.
constexpr float MAGIC_2P23 = 8388608.0f;

// Shape of the augmented moment tiles for B bands: the vector (x_0 .. x_{B-1}, 1)
// padded with zeros to BP (a multiple of 4) entries, cut into nb blocks of 4.
struct MomShape {
    int BA, BP, nb, nblk;
};

__host__ __device__ inline MomShape mom_shape(int B)
{
    MomShape s;
    s.BA = B + 1;
    s.BP = (s.BA + 3) & ~3;
    s.nb = s.BP / 4;
    s.nblk = s.nb * (s.nb + 1) / 2;
    return s;
}

// Index of the 4x4 block pair (bi, bj), bi <= bj, in row-major upper-triangle order.
__host__ __device__ inline int blk_index(int bi, int bj, int nb)
{
    return bi * nb - bi * (bi - 1) / 2 + (bj - bi);
}

// Device-resident model.  One per cva_model; written by the fit kernels and
// read by the projection kernels.  All matrices are [row][column].
struct DevModel {
    // ---- fit workspace: reset by the label scan of every fit ---------------
    // Exact integer moments of the augmented training vectors (x, 1) per
    // class: block pair (bi, bj), slot 4a + b holds sum x'_{4bi+a} x'_{4bj+b}.
    unsigned long long mom[MAXK][MAXBLK][16];
    int status;   // CVA_OK or the first device-side error of the current fit
    int fitted;   // 1 once a fit finished without error
    int r;        // eigenpairs taken from the reduced K x K problem
    int nvec;     // canonical vectors formed (columns of V)
    unsigned int cls_count[MAXK];   // training pixels per class
    unsigned int tile_ticket;       // CTAs of the label count done (the last one scans)

    // ---- fit results --------------------------------------------------------
    long long n[MAXK];          // training pixels per class
    double mu_c[MAXK][MAXB];    // class means
    double mu[MAXB];            // mean of all training pixels
    double Sw[MAXB][MAXB];      // within-class scatter
    double Sb[MAXB][MAXB];      // between-class scatter (formed on request from Mb)
    double Mb[MAXB][MAXK];      // sqrt(n_c) (mu_c - mu): Sb = Mb Mb^T
    double lam[MAXB];           // eigenvalues, descending
    double V[MAXB][MAXB];       // canonical vectors, V[b][j]

    // ---- FP32 projection coefficients ---------------------------------------
    //   y_j = sum_b Vf[b][j] ((2^23 + x_b) - shift[b]) - dofs[j]
    // with shift[b] = 2^23 + rint(mu_b) (the centring done exactly in FP32)
    // and dofs[j] = sum_b V[b][j] (mu_b - rint(mu_b)) rounded once.
    float Vf[MAXB][MAXB];
    float shift[MAXB];
    float dofs[MAXB];
    float train_range[2 * MAXB];  // (lo, hi) of each variate over the training pixels
    float work_range[2 * MAXB];   // scratch range for the two-pass global rescale

    // ---- FP64 form (CVA_PRECISION_FP64) -------------------------------------
    // (min, max) pairs of FP64 scores in the order-preserving 64-bit encoding
    // of ord_enc, so that integer atomics give the extremes.
    unsigned long long train_enc64[2 * MAXB];  // over the training pixels
    unsigned long long work_enc64[2 * MAXB];   // scratch for range passes

    // ---- order statistics of the third rescale ------------------------------
    unsigned int sel_prefix[2 * MAXB];  // known leading key bits of (lo, hi) of each variate
    unsigned int sel_rank[2 * MAXB];    // rank still to find among the keys with that prefix

    // ---- cluster-separation indices (Section 3) -----------------------------
    int ev_status;                      // CVA_OK or the evaluation's error
    unsigned long long ev_count[MAXK];  // labelled pixels per class
    double ev_sum[MAXK][MAXB];          // sums, then centroids
    double ev_scatter[MAXK];            // sums of distances, then scatters
    double ev_M[MAXK][MAXK];
    double ev_R[MAXK][MAXK];
    double ev_DI[MAXK][MAXK];
};

// -------------------------------------------------------------------------
// launchers (each defined in the translation unit that holds its kernel)
// -------------------------------------------------------------------------

// Row length (uint16 entries) of the gathered training matrix: the B band
// values, a 1, and zeros up to a multiple of 8 (16-byte rows).
__host__ __device__ inline int xtr_row(int B)
{
    return (B + 1 + 7) & ~7;
}

// Training-pixel passes: a reset, one pass over the labels writing every
// training pixel's index to its class's region of `list` (K regions of `cap`
// entries), then one pass that gathers every training pixel's bands into the
// class-major matrix `xtr` (`cap` rows of xtr_row(B)) and forms the exact
// moments from them in the same CTA.
cudaError_t launch_fit_moments(const uint16_t* cube, int B, long long P, const uint8_t* labels,
                               int K, DevModel* dm, uint16_t* xtr, unsigned int* list,
                               long long cap, int num_sms, cudaStream_t s);
cudaError_t launch_fit_finalize(DevModel* dm, int B, int K, int nvec, cudaStream_t s);
// The class moments as K x (B+1)(B+2)/2 int64 words (class-major, upper
// triangle of the augmented moment matrix, row-major), and back.
cudaError_t launch_moments_export(const DevModel* dm, int B, int K, long long* out, cudaStream_t s);
cudaError_t launch_moments_import(DevModel* dm, int B, int K, const long long* in, cudaStream_t s);
cudaError_t launch_train_range(int B, int K, const uint16_t* xtr, DevModel* dm, int nvec, int num_sms,
                               cudaStream_t s);
cudaError_t launch_scatter_sb(DevModel* dm, int B, int K, cudaStream_t s);
cudaError_t launch_range_init(float* range, int k, cudaStream_t s);
cudaError_t launch_project(const uint16_t* cube, int B, long long P, const DevModel* dm, int k,
                           float* out_f32, uint8_t* out_u8, const float* u8_range,
                           float* range_acc, int num_sms, cudaStream_t s);
cudaError_t launch_f32_range(const float* proj, int k, long long P, const DevModel* dm,
                             float* range_acc, int num_sms, cudaStream_t s);
cudaError_t launch_f32_to_u8(const float* proj, int k, long long P, const DevModel* dm,
                             const float* range, uint8_t* out, int num_sms, cudaStream_t s);

// Principal components of the pixels selected by `mask` (all when null):
// exact moments into class 0 of the model, then the B x B eigensolve.
cudaError_t launch_pca_moments(const uint16_t* cube, int B, long long P, const uint8_t* mask, DevModel* dm,
                               int num_sms, cudaStream_t s);
cudaError_t launch_pca_finalize(DevModel* dm, int B, int nvec, cudaStream_t s);

// Cluster-separation indices of the labelled classes of a k-band image
// (uint8 when f32 is null) into the model's ev_* fields.
cudaError_t launch_cluster_indices(const uint8_t* img_u8, const float* img_f32, int k, long long P,
                                   const uint8_t* labels, int K, DevModel* dm, int num_sms, cudaStream_t s);
// Interleaved RGB image from three of k planes (src: plane of R, G, B;
// invert: bit c inverts channel c).
cudaError_t launch_rgb_composite(const uint8_t* planes, long long P, int s0, int s1, int s2, int invert,
                                 uint8_t* rgb, int num_sms, cudaStream_t s);

// Third rescale: lo / hi of each of k projections with m values taken out of
// each tail (`hist`: 2 x 2048 words per variate, zero on entry and on exit).
cudaError_t launch_percentile_range(const float* proj, int k, long long P, long long m, DevModel* dm,
                                    unsigned int* hist, float* range_out, int num_sms, cudaStream_t s);
// 16-bit rescale of k float32 projections with the (lo, hi) pairs in `range`.
cudaError_t launch_f32_to_u16(const float* proj, int k, long long P, const float* range, uint16_t* out,
                              int num_sms, cudaStream_t s);

// FP64 form: the training range in FP64 (into dm->train_enc64), and the
// projection with FP64 coefficients and accumulation.  The 8-bit range comes
// from `u8_enc` (encoded FP64 pairs) when given, else from `u8_range`
// (float pairs); `enc_acc` receives the encoded extremes when given.
cudaError_t launch_train_range64(int B, int K, const uint16_t* xtr, DevModel* dm, int nvec, int num_sms,
                                 cudaStream_t s);
cudaError_t launch_enc_init(unsigned long long* enc, int k, cudaStream_t s);
cudaError_t launch_enc_to_float(const unsigned long long* enc, int k, float* out, cudaStream_t s);
cudaError_t launch_project64(const uint16_t* cube, int B, long long P, const DevModel* dm, int k,
                             float* out_f32, uint8_t* out_u8, const unsigned long long* u8_enc,
                             const float* u8_range, unsigned long long* enc_acc, int num_sms, cudaStream_t s);

// -------------------------------------------------------------------------
// batched form: many pages (cubes) in one set of launches
// -------------------------------------------------------------------------

// One page of a batch in device memory.  The first block is set from the
// host's page list by the set-up kernel; the second by the pool scan once the
// label counts are known.  Pages are kept in the caller's order, and the
// flattened work of the batch (label tiles, training rows, moment units,
// training-range items, projection items) is laid out page after page, so a
// work index maps to its page by a binary search on the page's first index.
struct PageDev {
    const uint16_t* cube;   // B x H x W
    const uint8_t* labels;  // H x W
    uint8_t* out;           // k x H x W
    double* eigvals;        // B doubles, or null
    DevModel* dm;           // the page's model block
    unsigned int* tiles;    // ntiles x (K + 1) words
    long long P;            // H W
    long long tile0;        // first label tile of the page
    long long item0;        // first projection item of the page
    int B, K, k, ntiles;
    int vec;                // labels 16-byte aligned
    int v8;                 // projected by the batched kernel (P % 8 == 0, aligned buffers)
    // ---- set on the device ----
    unsigned long long row0;    // first row of the page in the pooled training list
    unsigned long long xoff;    // uint16 offset of its rows in the pooled training matrix
    unsigned long long unit0;   // first moments unit (256 rows of one class)
    unsigned long long titem0;  // first training-range item (256 rows)
    unsigned long long nrows;   // training rows
};

// Totals of the device-side work of a batch (pool scan).
struct BatchTotals {
    unsigned long long rows, xtr, units, titems;
};

constexpr int BATCH_ROWS_PER_ITEM = 256;  // training rows per training-range item

// Largest page index p with key(pages[p]) <= v (pages sorted by key).
template <typename KeyFn>
__host__ __device__ inline int find_page(const PageDev* pages, int n, unsigned long long v, KeyFn key)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key(pages[mid]) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// `tile_page` / `item_page`: page of every label tile / projection item.
cudaError_t launch_batch_tile_count(const PageDev* pages, const int* tile_page, long long ntiles_total,
                                    cudaStream_t s);
cudaError_t launch_batch_tile_compact(const PageDev* pages, const int* tile_page, long long ntiles_total,
                                      unsigned int* list_pool, cudaStream_t s);
cudaError_t launch_batch_gather_moments(const PageDev* pages, int n, const BatchTotals* tot,
                                       const unsigned int* list_pool, uint16_t* xtr_pool, int max_b, int num_sms,
                                       cudaStream_t s);
cudaError_t launch_batch_finalize(const PageDev* pages, int n, cudaStream_t s);
cudaError_t launch_batch_train_range(const PageDev* pages, int n, const BatchTotals* tot,
                                     const uint16_t* xtr_pool, int max_k, int num_sms, cudaStream_t s);
cudaError_t launch_batch_project(const PageDev* pages, const int* item_page, long long it_begin, long long it_end,
                                 int groups_per_item, int grid, int k, cudaStream_t s);

// A pointer the GPU can read: device or managed memory, or host memory that
// is registered / mapped.  Plain pageable host memory is refused.
inline bool device_visible(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged ||
           (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr);
}

// -------------------------------------------------------------------------
// device helpers
// -------------------------------------------------------------------------

#ifdef __CUDACC__

// Record the first device-side error of a fit.
__device__ inline void set_status(DevModel* dm, int code)
{
    atomicCAS(&dm->status, 0, code);
}

// Float min / max on a float stored in global memory, via the ordering of
// IEEE-754 bit patterns: non-negative floats order like signed integers,
// negative floats order inversely like unsigned integers.
__device__ inline void atomic_min_float(float* addr, float v)
{
    if (!(v == v)) return;
    if (__float_as_int(v) >= 0) atomicMin(reinterpret_cast<int*>(addr), __float_as_int(v));
    else atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

__device__ inline void atomic_max_float(float* addr, float v)
{
    if (!(v == v)) return;
    if (__float_as_int(v) >= 0) atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
    else atomicMin(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

// Order-preserving map of a double onto a 64-bit unsigned integer (negative
// values: all bits inverted; others: sign bit set), and its inverse.
__host__ __device__ inline unsigned long long ord_enc_bits(unsigned long long b)
{
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline unsigned long long ord_dec_bits(unsigned long long u)
{
    return (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
}

// The low (sel = 0) or high (sel = 1) 16-bit half of `w` as the float 2^23 + x:
// the half's two bytes become the low mantissa bytes under the exponent byte
// 0x4B of 2^23 (one byte permute, exact).
__device__ inline float u16_lo_biased(uint32_t w)
{
    return __int_as_float(static_cast<int>(__byte_perm(w, 0x4B000000u, 0x7410)));
}
__device__ inline float u16_hi_biased(uint32_t w)
{
    return __int_as_float(static_cast<int>(__byte_perm(w, 0x4B000000u, 0x7432)));
}
__device__ inline float u16_biased(uint32_t x)
{
    return __int_as_float(static_cast<int>(0x4B000000u | x));
}

// 8-bit code of a projection value: floor(y * scale + off) clamped to 0..255,
// with scale = 255 / (hi - lo) and off = 1/2 - lo * scale, i.e.
// floor(255 (y - lo) / (hi - lo) + 1/2) up to FP32 rounding.
__device__ inline uint32_t to_code(float y, float scale, float off)
{
    const float t = fminf(fmaxf(__fmaf_rn(y, scale, off), 0.0f), 255.0f);
    return static_cast<uint32_t>(__float2int_rd(t));
}

// The scale that maps [lo, hi] onto [0, 255]; 0 when the range is empty.
__device__ inline float code_scale(float lo, float hi)
{
    float w = __fsub_rn(hi, lo);
    return (w > 0.0f && w < 3.0e38f) ? __fdiv_rn(255.0f, w) : 0.0f;
}

// The matching offset 1/2 - lo * scale.
__device__ inline float code_offset(float lo, float scale)
{
    return __fmaf_rn(-lo, scale, 0.5f);
}

#endif  // __CUDACC__

}  // namespace cva
