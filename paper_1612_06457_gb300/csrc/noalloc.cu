// noalloc.cu -- one entry point that runs a whole fit and the fused
// projection without allocating any device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory budget with no allocator hook, plug-ins of host
// applications that forbid device allocations after start-up, and
// latency-critical loops that must never enter the driver's allocator.  For
// them cva_fit_project_u8_noalloc keeps every piece of scratch memory the fit
// needs (the model block, the training list and the gathered training
// matrix) in one file-scope device array, sized for the
// limits below, which every GPU that loads this library holds until the
// process exits.  The caller passes only inputs and outputs.
//
// In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory: its device address is looked up with cudaGetSymbolAddress, once per
// device, by the first call made with that device current, and kept for the
// life of the process (a cudaDeviceReset reloads the module elsewhere, so the
// header rules out calls after one).
#include <mutex>

#include "cva_internal.cuh"

namespace {

using cva::DevModel;
using cva::device_visible;

constexpr long long NOALLOC_MAX_PIXELS = 1LL << 26;  // H W
constexpr long long NOALLOC_MAX_TRAIN = 1LL << 18;   // training pixels
constexpr size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t OFF_MODEL = 0;
constexpr size_t OFF_LIST = align256(OFF_MODEL + sizeof(DevModel));
constexpr size_t OFF_XTR = align256(OFF_LIST + sizeof(unsigned int) * NOALLOC_MAX_TRAIN * cva::MAXK);
constexpr size_t SCRATCH_BYTES =
    align256(OFF_XTR + sizeof(uint16_t) * NOALLOC_MAX_TRAIN * ((cva::MAXB + 1 + 7) & ~7));

static_assert(NOALLOC_MAX_PIXELS <= cva::MAX_PIXELS, "pixel limit above the ABI limit");

}  // namespace

// The scratch array (about 38 MB in device data, zero at module load).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[MAX_DEVICES] = {};
int g_num_sms[MAX_DEVICES] = {};

// Device address of the scratch array and the SM count for the current
// device, looked up once per device.
int scratch_for_current_device(unsigned char** addr, int* sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return CVA_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CVA_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CVA_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
        g_num_sms[dev] = n;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return CVA_OK;
}

}  // namespace

extern "C" int cva_fit_project_u8_noalloc(const uint16_t* cube, int B, int H, int W, const uint8_t* labels, int K,
                                          int k, uint8_t* out, double* eigvals, int* status, void* stream)
{
    if (!cube || !labels || !out) return CVA_ERR_INVALID_ARG;
    if (B < 1 || B > CVA_MAX_BANDS || K < 2 || K > CVA_MAX_CLASSES || H < 1 || W < 1) return CVA_ERR_INVALID_ARG;
    const long long P = static_cast<long long>(H) * W;
    if (P > NOALLOC_MAX_PIXELS) return CVA_ERR_INVALID_ARG;
    if (k < 1 || k > B) return CVA_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
    if (!device_visible(cube) || !device_visible(labels) || !device_visible(out)) return CVA_ERR_INVALID_ARG;
    unsigned char* base = nullptr;
    int sms = 0;
    const int rc = scratch_for_current_device(&base, &sms);
    if (rc != CVA_OK) return rc;
    DevModel* dm = reinterpret_cast<DevModel*>(base + OFF_MODEL);
    unsigned int* list = reinterpret_cast<unsigned int*>(base + OFF_LIST);
    uint16_t* xtr = reinterpret_cast<uint16_t*>(base + OFF_XTR);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // Every word that must start at zero (class counters, moments, status) is
    // cleared by the fit's first kernel, and every other byte is written
    // before it is read within a call, so the previous call's contents do not
    // leak into this one.
    cudaError_t e = cva::launch_fit_moments(cube, B, P, labels, K, dm, xtr, list, NOALLOC_MAX_TRAIN, sms, s);
    if (e == cudaSuccess) e = cva::launch_fit_finalize(dm, B, K, k, s);
    if (e == cudaSuccess) e = cva::launch_train_range(B, K, xtr, dm, k, sms, s);
    if (e == cudaSuccess) e = cva::launch_project(cube, B, P, dm, k, nullptr, out, dm->train_range, nullptr, sms, s);
    if (e == cudaSuccess && eigvals)
        e = cudaMemcpyAsync(eigvals, dm->lam, sizeof(double) * B, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, &dm->status, sizeof(int), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? CVA_OK : CVA_ERR_CUDA;
}
