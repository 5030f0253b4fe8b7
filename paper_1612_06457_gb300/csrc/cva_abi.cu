// cva_abi.cu -- the extern "C" entry points declared in include/cva.h.
//
// Host-side argument checks, then kernel launches on the caller's stream.
// The model object owns one DevModel block in device memory; the caller owns
// every cube, label, projection and image buffer.
#include <cstddef>
#include <cstring>
#include <new>

#include "cva_internal.cuh"

struct cva_model {
    int B;
    int K;
    int device;
    int num_sms;
    int nvec;
    int precision;
    int fit_nvec;        // canonical vectors formed by the last fit
    bool range64_valid;  // dm->train_enc64 belongs to the last fit
    bool pca;            // the last fit was a principal-component fit (no training range)
    cva::DevModel* dm;
    unsigned int* list;  // training-pixel indices, K class regions of cap entries
    uint16_t* xtr;       // gathered training matrix, cap rows of xtr_row(B)
    long long cap;       // training pixels `list` and `xtr` hold
    unsigned int* hist;  // order-statistic histograms, MAXB x 2 x 2048 words (zero between calls)
};

namespace {
constexpr size_t HIST_WORDS = static_cast<size_t>(cva::MAXB) * 2 * 2048;
}

namespace {

using cva::DevModel;
using cva::device_visible;

int from_cuda(cudaError_t e)
{
    return e == cudaSuccess ? CVA_OK : CVA_ERR_CUDA;
}

bool valid_dims(int B, int H, int W)
{
    if (B < 1 || B > CVA_MAX_BANDS || H < 1 || W < 1) return false;
    const long long P = static_cast<long long>(H) * W;
    return P < (1LL << 31);
}

// The FP64 training range of the last fit, formed on first use from the
// gathered training matrix (which stays valid until the next fit).
cudaError_t ensure_range64(cva_model* m, cudaStream_t s)
{
    if (m->range64_valid) return cudaSuccess;
    const cudaError_t e = cva::launch_train_range64(m->B, m->K, m->xtr, m->dm, m->fit_nvec, m->num_sms, s);
    if (e == cudaSuccess) m->range64_valid = true;
    return e;
}

int read_status(cva_model* m, cudaStream_t s, int* fitted)
{
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CVA_ERR_CUDA;
    int st[2] = {0, 0};
    e = cudaMemcpy(st, &m->dm->status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return CVA_ERR_CUDA;
    if (fitted) *fitted = st[1];
    return st[0];
}

}  // namespace

extern "C" {

const char* cva_strerror(int code)
{
    switch (code) {
        case CVA_OK: return "success";
        case CVA_ERR_INVALID_ARG: return "invalid argument";
        case CVA_ERR_EMPTY_CLASS: return "a class has no training pixel";
        case CVA_ERR_NOT_SPD: return "within-class scatter is not positive definite";
        case CVA_ERR_NO_CONVERGENCE: return "eigensolver did not converge";
        case CVA_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case CVA_ERR_CUDA: return "CUDA runtime error";
        case CVA_ERR_LABEL_RANGE: return "a label is above the class count";
        case CVA_ERR_NOT_FITTED: return "model not fitted";
        case CVA_ERR_CAPACITY: return "more training pixels than the model's index buffer holds";
        default: return "unknown error";
    }
}

int cva_model_create(int B, int K, cva_model** out)
{
    if (!out) return CVA_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1 || B > CVA_MAX_BANDS || K < 2 || K > CVA_MAX_CLASSES) return CVA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CVA_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CVA_ERR_CUDA;
    DevModel* dm = nullptr;
    unsigned int* list = nullptr;
    uint16_t* xtr = nullptr;
    unsigned int* hist = nullptr;
    const size_t cap = CVA_DEFAULT_TRAIN_CAPACITY;
    if (cudaMalloc(&dm, sizeof(DevModel)) != cudaSuccess) return CVA_ERR_CUDA;
    if (cudaMalloc(&list, sizeof(unsigned int) * cap * static_cast<size_t>(K)) != cudaSuccess ||
        cudaMalloc(&xtr, sizeof(uint16_t) * cap * cva::xtr_row(B)) != cudaSuccess ||
        cudaMalloc(&hist, sizeof(unsigned int) * HIST_WORDS) != cudaSuccess ||
        cudaMemset(dm, 0, sizeof(DevModel)) != cudaSuccess || cudaMemset(hist, 0, sizeof(unsigned int) * HIST_WORDS)) {
        cudaFree(dm);
        cudaFree(list);
        cudaFree(xtr);
        cudaFree(hist);
        return CVA_ERR_CUDA;
    }
    cva_model* m = new (std::nothrow) cva_model;
    if (!m) {
        cudaFree(dm);
        cudaFree(list);
        cudaFree(xtr);
        cudaFree(hist);
        return CVA_ERR_INVALID_ARG;
    }
    m->B = B;
    m->K = K;
    m->device = dev;
    m->num_sms = sms;
    m->nvec = B;
    m->precision = CVA_PRECISION_MIXED;
    m->fit_nvec = B;
    m->range64_valid = false;
    m->pca = false;
    m->dm = dm;
    m->list = list;
    m->xtr = xtr;
    m->hist = hist;
    m->cap = static_cast<long long>(cap);
    *out = m;
    return CVA_OK;
}

int cva_model_reserve(cva_model* m, int64_t max_train)
{
    if (!m || max_train < 1 || max_train >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
    if (max_train <= m->cap) return CVA_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return CVA_ERR_CUDA;
    unsigned int* list = nullptr;
    uint16_t* xtr = nullptr;
    if (cudaMalloc(&list, sizeof(unsigned int) * static_cast<size_t>(max_train) * m->K) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (cudaMalloc(&xtr, sizeof(uint16_t) * static_cast<size_t>(max_train) * cva::xtr_row(m->B)) != cudaSuccess) {
        cudaFree(list);
        return CVA_ERR_CUDA;
    }
    cudaFree(m->list);
    cudaFree(m->xtr);
    m->list = list;
    m->xtr = xtr;
    m->cap = max_train;
    return CVA_OK;
}

void cva_model_destroy(cva_model* m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->dm);
    cudaFree(m->list);
    cudaFree(m->xtr);
    cudaFree(m->hist);
    delete m;
}

int cva_set_precision(cva_model* m, int mode)
{
    if (!m || (mode != CVA_PRECISION_MIXED && mode != CVA_PRECISION_FP64)) return CVA_ERR_INVALID_ARG;
    m->precision = mode;
    return CVA_OK;
}

int cva_set_variates(cva_model* m, int nvec)
{
    if (!m || nvec < 1 || nvec > m->B) return CVA_ERR_INVALID_ARG;
    m->nvec = nvec;
    return CVA_OK;
}

int cva_fit(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K, cva_model* m,
            void* stream)
{
    if (!m || B != m->B || K != m->K || !valid_dims(B, H, W)) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || !device_visible(labels)) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    cudaError_t e =
        cva::launch_fit_moments(cube, B, P, labels, K, m->dm, m->xtr, m->list, m->cap, m->num_sms, s);
    if (e == cudaSuccess) e = cva::launch_fit_finalize(m->dm, B, K, m->nvec, s);
    if (e == cudaSuccess) e = cva::launch_train_range(B, K, m->xtr, m->dm, m->nvec, m->num_sms, s);
    m->fit_nvec = m->nvec;
    m->range64_valid = false;
    m->pca = false;
    if (e == cudaSuccess && m->precision == CVA_PRECISION_FP64) e = ensure_range64(m, s);
    return from_cuda(e);
}

int cva_fit_moments(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K, cva_model* m,
                    void* stream)
{
    if (!m || B != m->B || K != m->K || !valid_dims(B, H, W)) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || !device_visible(labels)) return CVA_ERR_INVALID_ARG;
    const long long P = static_cast<long long>(H) * W;
    const cudaError_t e = cva::launch_fit_moments(cube, B, P, labels, K, m->dm, m->xtr, m->list, m->cap,
                                                  m->num_sms, static_cast<cudaStream_t>(stream));
    m->range64_valid = false;
    m->pca = false;
    return from_cuda(e);
}

int cva_model_moments(cva_model* m, int64_t* moments, void* stream)
{
    if (!m || !device_visible(moments) || reinterpret_cast<uintptr_t>(moments) % 8 != 0) return CVA_ERR_INVALID_ARG;
    return from_cuda(cva::launch_moments_export(m->dm, m->B, m->K, reinterpret_cast<long long*>(moments),
                                                static_cast<cudaStream_t>(stream)));
}

int cva_fit_from_moments(cva_model* m, const int64_t* moments, void* stream)
{
    if (!m || !device_visible(moments) || reinterpret_cast<uintptr_t>(moments) % 8 != 0) return CVA_ERR_INVALID_ARG;
    if (m->precision != CVA_PRECISION_MIXED) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cva::launch_moments_import(m->dm, m->B, m->K, reinterpret_cast<const long long*>(moments), s);
    if (e == cudaSuccess) e = cva::launch_fit_finalize(m->dm, m->B, m->K, m->nvec, s);
    if (e == cudaSuccess) e = cva::launch_train_range(m->B, m->K, m->xtr, m->dm, m->nvec, m->num_sms, s);
    m->fit_nvec = m->nvec;
    m->range64_valid = false;
    m->pca = false;
    return from_cuda(e);
}

int cva_model_training_range(cva_model* m, float* range, void* stream)
{
    if (!m || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0) return CVA_ERR_INVALID_ARG;
    return from_cuda(cudaMemcpyAsync(range, m->dm->train_range, sizeof(float) * 2 * m->fit_nvec,
                                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
}

int cva_set_training_range(cva_model* m, const float* range, void* stream)
{
    if (!m || m->pca || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0)
        return CVA_ERR_INVALID_ARG;
    return from_cuda(cudaMemcpyAsync(m->dm->train_range, range, sizeof(float) * 2 * m->fit_nvec,
                                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)));
}

int cva_pca_fit(const uint16_t* cube, int B, int H, int W, const uint8_t* mask, cva_model* m, void* stream)
{
    if (!m || B != m->B || !valid_dims(B, H, W)) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || (mask && !device_visible(mask))) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    cudaError_t e = cva::launch_pca_moments(cube, B, P, mask, m->dm, m->num_sms, s);
    if (e == cudaSuccess) e = cva::launch_pca_finalize(m->dm, B, m->nvec, s);
    m->fit_nvec = m->nvec;
    m->range64_valid = false;
    m->pca = true;
    return from_cuda(e);
}

int cva_status(cva_model* m, void* stream)
{
    if (!m) return CVA_ERR_INVALID_ARG;
    return read_status(m, static_cast<cudaStream_t>(stream), nullptr);
}

int cva_model_get(cva_model* m, double* eigvals, double* V, double* mean, float* train_range, void* stream)
{
    if (!m) return CVA_ERR_INVALID_ARG;
    int fitted = 0;
    const int st = read_status(m, static_cast<cudaStream_t>(stream), &fitted);
    if (st != CVA_OK) return st;
    if (!fitted) return CVA_ERR_NOT_FITTED;
    const int B = m->B;
    const DevModel* dm = m->dm;
    if (eigvals && cudaMemcpy(eigvals, dm->lam, sizeof(double) * B, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (mean && cudaMemcpy(mean, dm->mu, sizeof(double) * B, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (train_range && m->precision == CVA_PRECISION_FP64 && !m->pca) {
        unsigned long long enc[2 * cva::MAXB];
        if (ensure_range64(m, static_cast<cudaStream_t>(stream)) != cudaSuccess ||
            cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess ||
            cudaMemcpy(enc, dm->train_enc64, sizeof(enc), cudaMemcpyDeviceToHost) != cudaSuccess)
            return CVA_ERR_CUDA;
        for (int i = 0; i < 2 * B; ++i) {
            const unsigned long long b = cva::ord_dec_bits(enc[i]);
            double d;
            std::memcpy(&d, &b, sizeof(d));
            train_range[i] = i < 2 * m->fit_nvec ? static_cast<float>(d) : 0.0f;
        }
    } else if (train_range &&
               cudaMemcpy(train_range, dm->train_range, sizeof(float) * 2 * B, cudaMemcpyDeviceToHost) != cudaSuccess) {
        return CVA_ERR_CUDA;
    }
    if (V && cudaMemcpy2D(V, sizeof(double) * B, dm->V, sizeof(double) * cva::MAXB, sizeof(double) * B, B,
                          cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    return CVA_OK;
}

int cva_model_get_scatter(cva_model* m, int64_t* counts, double* class_means, double* Sw, double* Sb,
                          void* stream)
{
    if (!m) return CVA_ERR_INVALID_ARG;
    int fitted = 0;
    const int st = read_status(m, static_cast<cudaStream_t>(stream), &fitted);
    if (st != CVA_OK) return st;
    if (!fitted) return CVA_ERR_NOT_FITTED;
    const int B = m->B, K = m->K;
    const DevModel* dm = m->dm;
    if (Sb && (cva::launch_scatter_sb(m->dm, B, K, static_cast<cudaStream_t>(stream)) != cudaSuccess ||
               cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess))
        return CVA_ERR_CUDA;
    if (counts && cudaMemcpy(counts, dm->n, sizeof(int64_t) * K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (class_means && cudaMemcpy2D(class_means, sizeof(double) * B, dm->mu_c, sizeof(double) * cva::MAXB,
                                    sizeof(double) * B, K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (Sw && cudaMemcpy2D(Sw, sizeof(double) * B, dm->Sw, sizeof(double) * cva::MAXB, sizeof(double) * B, B,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (Sb && cudaMemcpy2D(Sb, sizeof(double) * B, dm->Sb, sizeof(double) * cva::MAXB, sizeof(double) * B, B,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    return CVA_OK;
}

int cva_project(const uint16_t* cube, int B, int H, int W, cva_model* m, int k, float* out_f32,
                float* range_out, void* stream)
{
    if (!m || B != m->B || !valid_dims(B, H, W) || k < 1 || k > m->fit_nvec) return CVA_ERR_INVALID_ARG;
    if (!out_f32 && !range_out) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0 || reinterpret_cast<uintptr_t>(out_f32) % 4 != 0 ||
        reinterpret_cast<uintptr_t>(range_out) % 4 != 0)
        return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || (out_f32 && !device_visible(out_f32)) || (range_out && !device_visible(range_out)))
        return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    cudaError_t e = cudaSuccess;
    if (m->precision == CVA_PRECISION_FP64) {
        unsigned long long* acc = range_out ? m->dm->work_enc64 : nullptr;
        if (acc) e = cva::launch_enc_init(acc, k, s);
        if (e == cudaSuccess)
            e = cva::launch_project64(cube, B, P, m->dm, k, out_f32, nullptr, nullptr, nullptr, acc, m->num_sms, s);
        if (e == cudaSuccess && acc) e = cva::launch_enc_to_float(acc, k, range_out, s);
        return from_cuda(e);
    }
    if (range_out) e = cva::launch_range_init(range_out, k, s);
    if (e == cudaSuccess)
        e = cva::launch_project(cube, B, P, m->dm, k, out_f32, nullptr, nullptr, range_out, m->num_sms, s);
    return from_cuda(e);
}

int cva_to_u8(const float* proj, int k, int H, int W, int mode, const float* range, cva_model* m, uint8_t* out,
              void* stream)
{
    if (k < 1 || k > CVA_MAX_BANDS || H < 1 || W < 1 || static_cast<long long>(H) * W >= (1LL << 31))
        return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(proj) % 4 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(proj) || !device_visible(out)) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    cudaError_t e = cudaSuccess;
    const DevModel* dmc = m ? m->dm : nullptr;
    switch (mode) {
        case CVA_RANGE_GLOBAL:
            if (!m) return CVA_ERR_INVALID_ARG;
            e = cva::launch_range_init(m->dm->work_range, k, s);
            if (e == cudaSuccess) e = cva::launch_f32_range(proj, k, P, dmc, m->dm->work_range, m->num_sms, s);
            if (e == cudaSuccess) e = cva::launch_f32_to_u8(proj, k, P, dmc, m->dm->work_range, out, m->num_sms, s);
            break;
        case CVA_RANGE_TRAINING:
            if (!m || k > m->fit_nvec || m->pca) return CVA_ERR_INVALID_ARG;
            e = cva::launch_f32_to_u8(proj, k, P, dmc, m->dm->train_range, out, m->num_sms, s);
            break;
        case CVA_RANGE_GIVEN: {
            if (!range || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0)
                return CVA_ERR_INVALID_ARG;
            int sms = 0, dev = 0;
            if (m) sms = m->num_sms;
            else if (cudaGetDevice(&dev) != cudaSuccess ||
                     cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return CVA_ERR_CUDA;
            e = cva::launch_f32_to_u8(proj, k, P, dmc, range, out, sms, s);
            break;
        }
        default:
            return CVA_ERR_INVALID_ARG;
    }
    return from_cuda(e);
}

int cva_percentile_range(const float* proj, int k, int H, int W, double percent, cva_model* m, float* range_out,
                         void* stream)
{
    if (!m || k < 1 || k > CVA_MAX_BANDS || H < 1 || W < 1) return CVA_ERR_INVALID_ARG;
    const long long P = static_cast<long long>(H) * W;
    if (P >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
    const double scaled = percent * 100.0;
    if (!(scaled >= -1e-6 && scaled < 4999.5)) return CVA_ERR_INVALID_ARG;
    const long long bp = static_cast<long long>(scaled + 0.5);
    if (scaled - static_cast<double>(bp) > 1e-6 || static_cast<double>(bp) - scaled > 1e-6) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(proj) % 4 != 0 || reinterpret_cast<uintptr_t>(range_out) % 4 != 0)
        return CVA_ERR_INVALID_ARG;
    if (!device_visible(proj) || !device_visible(range_out)) return CVA_ERR_INVALID_ARG;
    const long long mt = (bp * P) / 10000;
    return from_cuda(cva::launch_percentile_range(proj, k, P, mt, m->dm, m->hist, range_out, m->num_sms,
                                                  static_cast<cudaStream_t>(stream)));
}

int cva_to_u16(const float* proj, int k, int H, int W, int mode, const float* range, cva_model* m, uint16_t* out,
               void* stream)
{
    if (k < 1 || k > CVA_MAX_BANDS || H < 1 || W < 1 || static_cast<long long>(H) * W >= (1LL << 31))
        return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(proj) % 4 != 0 || reinterpret_cast<uintptr_t>(out) % 2 != 0)
        return CVA_ERR_INVALID_ARG;
    if (!device_visible(proj) || !device_visible(out)) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    cudaError_t e = cudaSuccess;
    int sms = 0, dev = 0;
    if (m) sms = m->num_sms;
    else if (cudaGetDevice(&dev) != cudaSuccess ||
             cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CVA_ERR_CUDA;
    switch (mode) {
        case CVA_RANGE_GLOBAL:
            if (!m) return CVA_ERR_INVALID_ARG;
            e = cva::launch_range_init(m->dm->work_range, k, s);
            if (e == cudaSuccess) e = cva::launch_f32_range(proj, k, P, m->dm, m->dm->work_range, sms, s);
            if (e == cudaSuccess) e = cva::launch_f32_to_u16(proj, k, P, m->dm->work_range, out, sms, s);
            break;
        case CVA_RANGE_TRAINING:
            if (!m || k > m->fit_nvec || m->pca) return CVA_ERR_INVALID_ARG;
            e = cva::launch_f32_to_u16(proj, k, P, m->dm->train_range, out, sms, s);
            break;
        case CVA_RANGE_GIVEN:
            if (!range || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0)
                return CVA_ERR_INVALID_ARG;
            e = cva::launch_f32_to_u16(proj, k, P, range, out, sms, s);
            break;
        default:
            return CVA_ERR_INVALID_ARG;
    }
    return from_cuda(e);
}

int cva_cluster_indices(const void* image, int dtype, int k, int H, int W, const uint8_t* labels, int K, cva_model* m,
                        int64_t* counts, double* centroids, double* scatter, double* M, double* R, double* DI,
                        void* stream)
{
    if (!m || !image || !labels || k < 1 || k > CVA_MAX_BANDS || K < 1 || K > CVA_MAX_CLASSES || H < 1 || W < 1)
        return CVA_ERR_INVALID_ARG;
    if (dtype != CVA_IMAGE_U8 && dtype != CVA_IMAGE_F32) return CVA_ERR_INVALID_ARG;
    const long long P = static_cast<long long>(H) * W;
    if (P >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
    if (dtype == CVA_IMAGE_F32 && reinterpret_cast<uintptr_t>(image) % 4 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(image) || !device_visible(labels)) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevModel* dm = m->dm;
    cudaError_t e = cva::launch_cluster_indices(dtype == CVA_IMAGE_U8 ? static_cast<const uint8_t*>(image) : nullptr,
                                                dtype == CVA_IMAGE_F32 ? static_cast<const float*>(image) : nullptr,
                                                k, P, labels, K, dm, m->num_sms, s);
    if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CVA_ERR_CUDA;
    int st = 0;
    if (cudaMemcpy(&st, &dm->ev_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CVA_ERR_CUDA;
    if (st != CVA_OK) return st;
    if (counts) {
        unsigned long long c[cva::MAXK];
        if (cudaMemcpy(c, dm->ev_count, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return CVA_ERR_CUDA;
        for (int i = 0; i < K; ++i) counts[i] = static_cast<int64_t>(c[i]);
    }
    if (centroids && cudaMemcpy2D(centroids, sizeof(double) * k, dm->ev_sum, sizeof(double) * cva::MAXB,
                                  sizeof(double) * k, K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    if (scatter && cudaMemcpy(scatter, dm->ev_scatter, sizeof(double) * K, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CVA_ERR_CUDA;
    const double* tables[3] = {&dm->ev_M[0][0], &dm->ev_R[0][0], &dm->ev_DI[0][0]};
    double* outs[3] = {M, R, DI};
    for (int t = 0; t < 3; ++t)
        if (outs[t] && cudaMemcpy2D(outs[t], sizeof(double) * K, tables[t], sizeof(double) * cva::MAXK,
                                    sizeof(double) * K, K, cudaMemcpyDeviceToHost) != cudaSuccess)
            return CVA_ERR_CUDA;
    return CVA_OK;
}

int cva_rgb_composite(const uint8_t* planes, int k, int H, int W, const int* src, int invert, uint8_t* rgb,
                      void* stream)
{
    if (!planes || !src || !rgb || k < 1 || H < 1 || W < 1 || invert < 0 || invert > 7) return CVA_ERR_INVALID_ARG;
    const long long P = static_cast<long long>(H) * W;
    if (P >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
    for (int c = 0; c < 3; ++c)
        if (src[c] < 0 || src[c] >= k) return CVA_ERR_INVALID_ARG;
    if (!device_visible(planes) || !device_visible(rgb)) return CVA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CVA_ERR_CUDA;
    return from_cuda(cva::launch_rgb_composite(planes, P, src[0], src[1], src[2], invert, rgb, sms,
                                               static_cast<cudaStream_t>(stream)));
}

int cva_project_u8(const uint16_t* cube, int B, int H, int W, cva_model* m, int k, int mode, const float* range,
                   uint8_t* out, void* stream)
{
    if (!m || B != m->B || !valid_dims(B, H, W) || k < 1 || k > m->fit_nvec) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || !device_visible(out)) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = static_cast<long long>(H) * W;
    DevModel* dm = m->dm;
    cudaError_t e = cudaSuccess;
    if (mode == CVA_RANGE_TRAINING && m->pca) return CVA_ERR_INVALID_ARG;
    if (m->precision == CVA_PRECISION_FP64) {
        switch (mode) {
            case CVA_RANGE_TRAINING:
                e = ensure_range64(m, s);
                if (e == cudaSuccess)
                    e = cva::launch_project64(cube, B, P, dm, k, nullptr, out, dm->train_enc64, nullptr, nullptr,
                                              m->num_sms, s);
                break;
            case CVA_RANGE_GIVEN:
                if (!range || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0)
                    return CVA_ERR_INVALID_ARG;
                e = cva::launch_project64(cube, B, P, dm, k, nullptr, out, nullptr, range, nullptr, m->num_sms, s);
                break;
            case CVA_RANGE_GLOBAL:
                e = cva::launch_enc_init(dm->work_enc64, k, s);
                if (e == cudaSuccess)
                    e = cva::launch_project64(cube, B, P, dm, k, nullptr, nullptr, nullptr, nullptr, dm->work_enc64,
                                              m->num_sms, s);
                if (e == cudaSuccess)
                    e = cva::launch_project64(cube, B, P, dm, k, nullptr, out, dm->work_enc64, nullptr, nullptr,
                                              m->num_sms, s);
                break;
            default:
                return CVA_ERR_INVALID_ARG;
        }
        return from_cuda(e);
    }
    switch (mode) {
        case CVA_RANGE_TRAINING:
            e = cva::launch_project(cube, B, P, dm, k, nullptr, out, dm->train_range, nullptr, m->num_sms, s);
            break;
        case CVA_RANGE_GIVEN:
            if (!range || !device_visible(range) || reinterpret_cast<uintptr_t>(range) % 4 != 0)
                return CVA_ERR_INVALID_ARG;
            e = cva::launch_project(cube, B, P, dm, k, nullptr, out, range, nullptr, m->num_sms, s);
            break;
        case CVA_RANGE_GLOBAL:
            e = cva::launch_range_init(dm->work_range, k, s);
            if (e == cudaSuccess)
                e = cva::launch_project(cube, B, P, dm, k, nullptr, nullptr, nullptr, dm->work_range, m->num_sms, s);
            if (e == cudaSuccess)
                e = cva::launch_project(cube, B, P, dm, k, nullptr, out, dm->work_range, nullptr, m->num_sms, s);
            break;
        default:
            return CVA_ERR_INVALID_ARG;
    }
    return from_cuda(e);
}

}  // extern "C"
