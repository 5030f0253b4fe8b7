/*
 * cva.h -- C ABI of the GB300 (sm_103a) Canonical Variates Analysis library.
 *
 * The library fits Canonical Variates Analysis (CVA) to the labelled training
 * pixels of a multispectral cube and projects every pixel of the cube onto
 * the top canonical variates, rescaled to 8-bit images, as described in
 * arXiv 1612.06457 (Arsene, Church, Dickinson), Section 2 (the method and
 * the three rescales) and Section 4 (the generalized symmetric-definite
 * eigenproblem solved by GSL, and the eigenvector sign ambiguity).
 *
 * Contents: models and the fit (cva_model_*, cva_fit, cva_set_variates,
 * cva_set_precision, getters); projections and rescales (cva_project,
 * cva_to_u8, cva_project_u8, the third rescale's cva_percentile_range,
 * cva_to_u16); principal components (cva_pca_fit); Section 3's evaluation
 * indices and the colour composite (cva_cluster_indices, cva_rgb_composite);
 * the batched form for many pages (cva_batch_*, cva_fit_project_batched,
 * cva_project_batched); and an allocation-free fit + projection
 * (cva_fit_project_u8_noalloc).
 *
 * Conventions shared by every call:
 *   - Data pointers marked "device" must point to device memory of the
 *     current CUDA device; the caller owns them.  Host pointers are marked
 *     "host".  The library owns only its model objects.
 *   - cube: uint16, band-sequential (band-major), B x H x W, band b of pixel
 *     p = y W + x at cube[b H W + p].  Band 0 is the first band of the stack.
 *   - labels: uint8, H x W, 0 = not a training pixel, c + 1 = training pixel
 *     of class c (0 <= c < K).
 *   - projections: float32 k x H x W (variate-major); 8-bit images: uint8
 *     k x H x W; ranges: 2 k float32 as (lo_0, hi_0, lo_1, hi_1, ...).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call that takes a stream is asynchronous on it unless
 *     its comment says it synchronizes.
 *   - Return value: CVA_OK (0) or a negative CVA_ERR_* code.  Argument errors
 *     are detected on the host and returned at once, before any launch.
 *     Errors found on the device (an empty class, a label above K, Sw not
 *     positive definite, no convergence) are written to the model's status
 *     word; cva_status() and cva_model_get() return them.  Projections from
 *     a model whose fit failed leave their outputs untouched.
 *   - Limits: 1 <= B <= CVA_MAX_BANDS, 2 <= K <= CVA_MAX_CLASSES,
 *     1 <= H, W and H W < 2^31, 1 <= k <= B.
 */
#ifndef CVA_H_
#define CVA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CVA_MAX_BANDS 32
#define CVA_MAX_CLASSES 16

#define CVA_OK 0
#define CVA_ERR_INVALID_ARG (-1)    /* bad size, pointer, mode or alignment */
#define CVA_ERR_EMPTY_CLASS (-2)    /* a class has no training pixel */
#define CVA_ERR_NOT_SPD (-3)        /* within-class scatter not positive definite */
#define CVA_ERR_NO_CONVERGENCE (-4) /* the eigenvector refinement did not converge */
#define CVA_ERR_TIMEOUT (-5)        /* reserved: no kernel of this library waits on another */
#define CVA_ERR_CUDA (-6)           /* a CUDA runtime call failed */
#define CVA_ERR_LABEL_RANGE (-7)    /* a label is above K */
#define CVA_ERR_NOT_FITTED (-8)     /* the model has not been fitted */
#define CVA_ERR_CAPACITY (-9)       /* more training pixels than the model can hold */

/* Which range maps a projection onto 0..255 (Section 2 gives the first two). */
typedef enum {
    CVA_RANGE_GLOBAL = 0,   /* min / max over every pixel of the projection */
    CVA_RANGE_TRAINING = 1, /* min / max over the training pixels' scores */
    CVA_RANGE_GIVEN = 2     /* a caller-supplied range */
} cva_range_mode;

/* Arithmetic of the projection and of the training-score range.  The fit is
 * the same in both: class moments from BF16 hi/lo split pixel values
 * (x = 256 hi + lo, both exact in BF16) on the tensor cores with FP32
 * accumulation, exact because every partial sum stays below 2^24 and is
 * merged in 64-bit integers; scatter matrices rounded once to FP64;
 * Cholesky, eigensolve and coefficients in double-float (about 48 bits) and
 * published as FP64. */
typedef enum {
    /* Default.  Projection in FP32: exact centring on the integer part of
     * the mean, FP32 coefficients and accumulation.  HBM-bound. */
    CVA_PRECISION_MIXED = 0,
    /* Projection and training range with FP64 coefficients, centring and
     * accumulation; 8-bit codes computed in FP64.  Bound by the FP64 pipe,
     * several times slower; the plain form the mixed one is measured
     * against.  cva_to_u8 is FP32 in both modes (its input is FP32). */
    CVA_PRECISION_FP64 = 1
} cva_precision_mode;

typedef struct cva_model cva_model;

/* Create a model for B bands and K classes on the current CUDA device.  Owns
 * until cva_model_destroy: a device block of about 150 KB, a 512 KB
 * histogram block for cva_percentile_range, and, with room for
 * CVA_DEFAULT_TRAIN_CAPACITY training pixels (see cva_model_reserve), the
 * gathered training matrix of 2 ((B + 8) & ~7) bytes per training pixel and
 * a training-pixel index list of 4 K bytes per training pixel.  *out is set to
 * NULL on error.  Not stream-ordered: allocates with cudaMalloc, so call it
 * outside stream capture. */
#define CVA_DEFAULT_TRAIN_CAPACITY (1 << 22)
int cva_model_create(int B, int K, cva_model** out);

/* Make room for up to `max_train` labelled training pixels per fit (a fit
 * with more sets CVA_ERR_CAPACITY in the device status).  Synchronizes the
 * device and reallocates; call it outside stream capture. */
int cva_model_reserve(cva_model* m, int64_t max_train);

/* Free the model (synchronizes the device first).  NULL is a no-op. */
void cva_model_destroy(cva_model* m);

/* Select CVA_PRECISION_MIXED (default) or CVA_PRECISION_FP64 for the
 * following calls.  May change between a fit and its projections: the FP64
 * training range is formed by the fit in FP64 mode, else by the first call
 * that needs it (from the fit's gathered training pixels).  Host-side only. */
int cva_set_precision(cva_model* m, int mode);

/* Number of canonical vectors, with their training-score ranges, that each
 * following fit forms: 1 <= nvec <= B (default B).  Projections take
 * k <= nvec.  The first min(K-1, B) vectors solve the eigenproblem with
 * non-zero eigenvalues; any further ones complete the basis of the
 * eigenvalue-0 space (V^T Sw V = I still holds) and are not unique. */
int cva_set_variates(cva_model* m, int nvec);

/* Fit (Section 2: within-class and between-class scatter of the labelled
 * training pixels and their eigenanalysis; Section 4: Sb v = lambda Sw v).
 *   cube   device, B x H x W uint16 (2-byte aligned)
 *   labels device, H x W uint8 (0 = unlabelled, c + 1 = class c)
 * Results stay in the model on the device: eigenvalues lambda in descending
 * order, eigenvectors V with V^T Sw V = I and the largest-magnitude
 * component of each positive (lowest band on a tie), the training mean, and
 * the training-score range of each variate.  Sw and Sb are unnormalised
 * sums of squares and cross-products.  Forms the number of vectors set by
 * cva_set_variates.  Only kernel launches on `stream`: no host
 * synchronization and no allocation.  The labelled pixels are counted,
 * gathered class by class into the model's training matrix, and their exact
 * integer moments accumulated; errors (a label above K, an empty class, more
 * training pixels than the matrix holds, Sw not positive definite) go to the
 * device status. */
int cva_fit(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K,
            cva_model* m, void* stream);

/* ---- One page split over several GPUs ------------------------------------
 * Section 2's scatter matrices are sums over the training pixels, so a page
 * can be cut into parts (e.g. bands of rows, one per GPU) whose exact integer
 * class moments add up to the page's.  Each part's process calls
 * cva_fit_moments on its part, exports the moments with cva_model_moments,
 * sums them over all parts (an int64 all-reduce: exact, so the merged fit is
 * bit-identical to cva_fit on the whole page), and calls
 * cva_fit_from_moments with the sum; that fit also forms the training-score
 * range of its own part's training pixels, which cva_model_training_range
 * exports; the parts' ranges merge by min / max (of the lo and of the hi
 * entries) and cva_set_training_range installs the merged range, after which
 * cva_project_u8 with CVA_RANGE_TRAINING on each part gives the page's
 * 8-bit image part by part.  Every call is asynchronous on `stream`.
 *
 * Words of the moment array: K classes of (B+1)(B+2)/2 int64 each. */
#define CVA_MOMENT_WORDS(B, K) ((K) * ((B) + 1) * ((B) + 2) / 2)

/* The class moments of the labelled pixels of a cube (or of one part of a
 * page): for each class c the sums over its training pixels of x'_a x'_b,
 * a <= b, with x' = (x_0 .. x_{B-1}, 1), so that the count n_c and the band
 * sums s_c are among them.  Kept in the model (and the part's training pixels
 * in its training matrix); no eigensolve.  Arguments and device errors as for
 * cva_fit. */
int cva_fit_moments(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K, cva_model* m,
                    void* stream);

/* Copy the model's class moments to `moments` (device, CVA_MOMENT_WORDS(B, K)
 * int64, 8-byte aligned): class c's entry (a, b), a <= b <= B, at
 * c (B+1)(B+2)/2 + a (B+1) - a (a-1)/2 + (b - a). */
int cva_model_moments(cva_model* m, int64_t* moments, void* stream);

/* Replace the model's class moments by `moments` (device, layout of
 * cva_model_moments; e.g. the sum over all parts of a page) and finish the
 * fit from them: means, Sw, Sb, the eigensolve and the canonical vectors as
 * in cva_fit, then the training-score range of the training pixels of the
 * model's last cva_fit_moments (its own part).  CVA_PRECISION_MIXED only.
 * Device errors go to the status word as for cva_fit. */
int cva_fit_from_moments(cva_model* m, const int64_t* moments, void* stream);

/* Copy out (device, 2 nvec float32, (lo, hi) pairs) the model's
 * training-score range, or install a range in its place (e.g. the min / max
 * merge of every part's range). */
int cva_model_training_range(cva_model* m, float* range, void* stream);
int cva_set_training_range(cva_model* m, const float* range, void* stream);

/* Principal components instead of canonical variates (Section 2: the
 * unsupervised PCA of the whole page -- subtract the mean, form the
 * covariance matrix, take its eigenvectors, orthonormal -- and, with a mask,
 * of the folio cropped out of the page or of chosen points).  The model's
 * eigenvalues become those of the sample covariance
 * C = sum_p (x_p - mu)(x_p - mu)^T / (N - 1) over the N selected pixels, in
 * descending order, and V its orthonormal eigenvectors (V^T V = I, same sign
 * convention), mean the mean of the selected pixels.  The moments are exact
 * (64-bit integer sums from BF16 hi/lo split values on the tensor cores),
 * the eigensolve as for cva_fit.  Afterwards cva_project, cva_project_u8 and
 * cva_to_u8 / cva_to_u16 work with CVA_RANGE_GLOBAL and CVA_RANGE_GIVEN
 * (there are no training pixels: CVA_RANGE_TRAINING is refused), and
 * cva_model_get_scatter returns counts[0] = N, class_means[0] = mean,
 * Sw = C and Sb = 0.  The model's K is not used.
 *   cube   device, B x H x W uint16 (B = the model's band count)
 *   mask   device, H x W uint8 (nonzero = pixel used), or NULL for all
 * Device errors: CVA_ERR_EMPTY_CLASS when fewer than 2 pixels are selected.
 * Asynchronous; allocates nothing. */
int cva_pca_fit(const uint16_t* cube, int B, int H, int W, const uint8_t* mask, cva_model* m,
                void* stream);

/* Synchronize `stream` and return the model's device status (CVA_OK or the
 * first device-side error of the last fit). */
int cva_status(cva_model* m, void* stream);

/* Copy the fitted model to host memory; synchronizes `stream`.  Any pointer
 * may be NULL to skip that output.
 *   eigvals      host, B doubles (descending; 0 beyond the first min(K-1, B))
 *   V            host, B x B doubles, row-major, column j = canonical vector j
 *                (columns j >= nvec, see cva_set_variates, are 0)
 *   mean         host, B doubles (mean of all training pixels)
 *   train_range  host, 2 B floats: training-score (lo, hi) of each variate
 *                in the current precision mode (FP64 mode: rounded to
 *                float); undefined for j >= nvec
 * Returns the model's device status, or CVA_ERR_NOT_FITTED. */
int cva_model_get(cva_model* m, double* eigvals, double* V, double* mean, float* train_range,
                  void* stream);

/* Copy the fit's intermediate statistics to host memory; synchronizes.
 *   counts       host, K int64 training pixels per class
 *   class_means  host, K x B doubles
 *   Sw, Sb       host, B x B doubles each (row-major)
 * Any pointer may be NULL.  Returns the model's device status. */
int cva_model_get_scatter(cva_model* m, int64_t* counts, double* class_means, double* Sw,
                          double* Sb, void* stream);

/* Projection (Section 2: the canonical coefficients multiplied with the band
 * images): out_f32[j][p] = sum_b V[b][j] (x_b[p] - mean_b) for j < k.
 *   out_f32   device, k x H x W float32, or NULL
 *   range_out device, 2 k float32, or NULL: receives the (lo, hi) of each
 *             projection over all pixels (the first rescale's range)
 * At least one of out_f32 / range_out must be non-NULL. */
int cva_project(const uint16_t* cube, int B, int H, int W, cva_model* m, int k,
                float* out_f32, float* range_out, void* stream);

/* Rescale projections to 8 bits (Section 2):
 * out = clamp(floor(255 (y - lo) / (hi - lo) + 1/2), 0, 255), 0 if hi <= lo.
 *   proj  device, k x H x W float32 from cva_project
 *   mode  CVA_RANGE_GLOBAL (range computed here from proj, into the model's
 *         scratch range), CVA_RANGE_TRAINING (range from the model), or
 *         CVA_RANGE_GIVEN (range = device 2 k float32)
 *   m     required for CVA_RANGE_GLOBAL and CVA_RANGE_TRAINING; may be NULL
 *         for CVA_RANGE_GIVEN
 *   out   device, k x H x W uint8 */
int cva_to_u8(const float* proj, int k, int H, int W, int mode, const float* range,
              cva_model* m, uint8_t* out, void* stream);

/* The third rescale's range (Section 2: the 0.01, 0.1, 1 or 5 percentiles of
 * the projected data taken out before the same linear rescale).  With p =
 * `percent` and m = floor(p P / 100) values taken out at EACH end of every
 * projection, range_out[2 j] is the (m+1)-th smallest and range_out[2 j + 1]
 * the (m+1)-th largest value of proj[j] (exact order statistics of the
 * float32 values).  Feed it to cva_to_u8 / cva_to_u16 with CVA_RANGE_GIVEN;
 * pixels outside the range clamp to 0 and the top code.
 *   proj       device, k x H x W float32 (4-byte aligned)
 *   percent    a multiple of 0.01 in [0, 50); 0 gives the global range
 *   m          any model on this device: its scratch (a 512 KB histogram
 *              block and 256 bytes of state) is used, so calls sharing a
 *              model must not overlap on the GPU
 *   range_out  device, 2 k float32
 * Three passes over proj, asynchronous on `stream`. */
int cva_percentile_range(const float* proj, int k, int H, int W, double percent, cva_model* m,
                         float* range_out, void* stream);

/* 16-bit image of the same rescale (the paper's C tool writes 8- and 16-bit
 * images): out = clamp(floor(65535 (y - lo) / (hi - lo) + 1/2), 0, 65535),
 * 0 if hi <= lo.  Arguments as for cva_to_u8; out is device k x H x W uint16
 * (2-byte aligned). */
int cva_to_u16(const float* proj, int k, int H, int W, int mode, const float* range,
               cva_model* m, uint16_t* out, void* stream);

/* Element types of an image given to cva_cluster_indices. */
#define CVA_IMAGE_U8 0   /* uint8 planes (the 8-bit images) */
#define CVA_IMAGE_F32 1  /* float32 planes (the projections) */

/* Cluster-separation indices of the labelled classes in a k-band image
 * (Section 3, eqs. 1-5, with p = 2): for each class c its labelled pixel
 * count T_c, centroid A_c and scatter S_c (mean Euclidean distance of its
 * pixels to A_c, eq. 1); for each pair the centroid distance M_ij (eq. 2),
 * the Davies-Bouldin ratio R_ij = (S_i + S_j) / M_ij (eq. 3) and the Dunn
 * index DI_ij = (M_ij - S_i - S_j) / max(S_i, S_j) (eq. 5).  Diagonals are 0;
 * R is +inf when two centroids coincide and DI when both scatters are 0.
 *   image   device, k x H x W planes of `dtype`
 *   labels  device, H x W uint8 (0 = not used, c + 1 = class c)
 *   m       any model on this device (its evaluation scratch is used)
 *   counts (K), centroids (K x k), scatter (K), M, R, DI (K x K): host
 *           outputs, row-major, each may be NULL
 * Synchronizes `stream`.  Returns CVA_ERR_LABEL_RANGE for a label above K
 * and CVA_ERR_EMPTY_CLASS for a class without pixels. */
int cva_cluster_indices(const void* image, int dtype, int k, int H, int W, const uint8_t* labels, int K,
                        cva_model* m, int64_t* counts, double* centroids, double* scatter, double* M,
                        double* R, double* DI, void* stream);

/* Colour image from three of k 8-bit images (Section 2 / Figure 5: three
 * grayscale images as the red, green and blue channels, the one with the
 * clearest undertext usually in green; Figure 5 also inverts channels):
 * rgb[3 p + c] = planes[src[c]][p], or 255 minus it when bit c of `invert`
 * is set.
 *   planes  device, k x H x W uint8;  src  host, 3 plane indices (R, G, B)
 *   rgb     device, H x W x 3 uint8 (interleaved)
 * Asynchronous; one pass. */
int cva_rgb_composite(const uint8_t* planes, int k, int H, int W, const int* src, int invert, uint8_t* rgb,
                      void* stream);

/* Fused projection and 8-bit rescale: one pass over the cube for
 * CVA_RANGE_TRAINING and CVA_RANGE_GIVEN, two passes (range, then
 * projection) for CVA_RANGE_GLOBAL.
 *   range device, 2 k float32 for CVA_RANGE_GIVEN, else NULL
 *   out   device, k x H x W uint8 */
int cva_project_u8(const uint16_t* cube, int B, int H, int W, cva_model* m, int k, int mode,
                   const float* range, uint8_t* out, void* stream);

/* Fit and fused projection to 8 bits in one call that allocates no device
 * memory (the paper has no counterpart: this serves callers that cannot
 * allocate, e.g. code running inside another framework's memory budget,
 * application plug-ins that forbid device allocations after start-up, or
 * loops that must never enter the driver's allocator).
 * Does what cva_fit followed by cva_project_u8 with CVA_RANGE_TRAINING does
 * (the same kernels), forming k canonical vectors.  All scratch memory (about
 * 38 MB) is one array in the library's device data, which every GPU that
 * loads the library holds until the process exits.
 *   cube, labels  device, as for cva_fit
 *   k             variates to project, 1 <= k <= B
 *   out           device, k x H x W uint8
 *   eigvals       device, B doubles, or NULL: the eigenvalues
 *   status        device, one int, or NULL: CVA_OK or the device-side error
 *                 of this call; on an error `out` is not written and
 *                 `eigvals` holds no meaningful values
 * Limits: H W <= 2^26 pixels (host check, CVA_ERR_INVALID_ARG) and at most
 * 2^18 training pixels (device check, CVA_ERR_CAPACITY in *status).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: do not call this entry point on a device after cudaDeviceReset
 * (or any other teardown of its primary context), since the kept address no
 * longer names the array then.  Every call shares the one array: calls that
 * overlap on the GPU (other streams, other host threads) race.  Calls are
 * asynchronous on `stream`. */
int cva_fit_project_u8_noalloc(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K,
                               int k, uint8_t* out, double* eigvals, int* status, void* stream);

/* ---- Batched form -------------------------------------------------------
 * Many pages (cubes of uneven size, band count and class count) fitted and
 * projected to 8 bits with the training-score range (CVA_RANGE_TRAINING), in
 * one fixed sequence of about ten launches whatever the page count, so that a
 * whole batch can be captured as one CUDA graph.  Each page is the problem of
 * Section 2 on its own (its own classes, scatter matrices and eigenvectors);
 * the results equal cva_fit + cva_project_u8 on each page. */
#define CVA_MAX_BATCH_PAGES 4096
#define CVA_MAX_BATCH_VARIATES 8

typedef struct {
    const uint16_t* cube;  /* device, B x H x W (2-byte aligned) */
    const uint8_t* labels; /* device, H x W: 0 = unlabelled, c + 1 = class c */
    uint8_t* out;          /* device, k x H x W */
    double* eigvals;       /* device, B doubles, or NULL */
    int B, H, W;           /* 1 <= B <= CVA_MAX_BANDS, H W < 2^31 */
    int K;                 /* 2 <= K <= CVA_MAX_CLASSES */
    int k;                 /* variates, 1 <= k <= min(B, CVA_MAX_BATCH_VARIATES) */
} cva_page;

typedef struct cva_batch cva_batch;

/* Workspace for batches of up to max_pages pages holding up to max_pixels
 * pixels in all and up to max_train training pixels in all (< 2^32).  Owns
 * until cva_batch_destroy: one model block (~150 KB) per page, a tile
 * workspace of 68 bytes per 16384 pixels, and pooled training storage of 84
 * bytes per training pixel.  Allocates with cudaMalloc: call it outside stream
 * capture.  *out is set to NULL on error. */
int cva_batch_create(int max_pages, int64_t max_pixels, int64_t max_train, cva_batch** out);
void cva_batch_destroy(cva_batch* b);

/* Fit and project every page of `pages` (host array of n descriptors, read
 * during the call only).  Asynchronous on `stream`; allocates nothing.
 * Host checks (CVA_ERR_INVALID_ARG): n, every page's sizes, device-visible
 * buffers; CVA_ERR_CAPACITY when the pages' pixels exceed the workspace.  A
 * page whose labels exceed K, whose class is empty, whose S_w is not positive
 * definite, or that overflows the pooled training storage fails alone: its
 * output is left untouched and cva_batch_status reports it.  Calls on one
 * workspace must not overlap on the GPU. */
int cva_fit_project_batched(cva_batch* b, const cva_page* pages, int n, void* stream);

/* The fit alone: every page's fit and training-score range, no projection
 * (cva_project_batched then projects).  Splitting the two lets a caller run
 * the projection of one batch while the next batch is fitted, e.g. the fits
 * on a high-priority stream and the projections on a low-priority one.
 * Asynchronous; allocates nothing. */
int cva_fit_batched(cva_batch* b, const cva_page* pages, int n, void* stream);

/* The projection pass alone: project every page again with the models of
 * the last cva_fit_project_batched (or cva_fit_batched) on this workspace, which must have been
 * given the same pages in the same order (same shapes and classes; the cube
 * contents may differ, e.g. the same pages imaged again).  Asynchronous;
 * allocates nothing. */
int cva_project_batched(cva_batch* b, const cva_page* pages, int n, void* stream);

/* Synchronize `stream` and copy each page's status of the last batch into
 * status (host, n ints; CVA_OK, a device-side error, or CVA_ERR_NOT_FITTED).
 * Returns CVA_OK or the first page's error. */
int cva_batch_status(cva_batch* b, int n, int* status, void* stream);

/* Autotuner of the batched projection: runs the batch once, then times the
 * projection pass with each work-item size (1, 2, 4, 8, 16 or 32 groups of
 * 2048 pixels) and grid (two persistent CTAs per SM, each on a contiguous run
 * of items; or one CTA per item) on
 * `pages` and keeps the fastest for later calls on this workspace.
 * Synchronizes `stream`; call it outside stream capture.  chosen (host, 2
 * ints, or NULL) receives the groups per item and the CTAs per SM (0 = one
 * per item). */
int cva_batch_tune(cva_batch* b, const cva_page* pages, int n, void* stream, int* chosen);

/* Human-readable text of a CVA_* code (static storage). */
const char* cva_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* CVA_H_ */
