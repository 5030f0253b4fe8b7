// batch.cu -- the batched form: fit and fused 8-bit projection of many pages
// (cubes of uneven size, band count and class count) in one fixed sequence of
// launches, so that a whole batch is one CUDA graph.
//
// A single page's fit is a chain of small, latency-bound passes (tens of
// microseconds each on a 16 M-pixel page, dominated by the single-CTA
// eigensolve); running 64 pages one after another would leave the GPU mostly
// idle.  Here every pass runs once for the whole batch over the flattened
// work of all pages (label tiles, pooled training rows, moment units, one
// eigensolve CTA per page side by side, training-range items, projection
// items), each work index mapped back to its page by a binary search on the
// pages' first indices.
//
// Launch sequence of one batch:
//   kb_setup           page table from the host's list (kernel parameters,
//                      so a captured graph holds its own copy)
//   kb_tile_count      label counts of every tile of every page; each page's
//                      last CTA takes that page's prefix sums
//   kb_pool_scan       one CTA: prefix sums over pages of the training rows,
//                      pooled matrix words, moment units and range items;
//                      capacity check of the pooled training storage
//   kb_tile_compact    class-major training lists, one per page, in the pool
//   kb_gather_moments  the pooled training matrix, gathered unit by unit,
//                      and its exact moments on the tensor cores
//   kb_fit_finalize    one CTA per page
//   kb_train_range<k>  training-score ranges
//   kb_project_v8<k>   fused projection + 8-bit rescale (persistent)
// Pages whose pixel count is not a multiple of 8 or whose buffers are not
// aligned for 16-byte loads are projected by the single-page kernels after
// the batched pass.
#include <cstring>
#include <new>

#include "cva_internal.cuh"

namespace {

using cva::BatchTotals;
using cva::DevModel;
using cva::device_visible;
using cva::PageDev;

constexpr int SETUP_CHUNK = 24;          // pages per set-up launch (3 KB of kernel parameters)
constexpr int XTR_POOL_ROW = 40;         // widest training row (32 bands + 1, padded to 8), uint16
constexpr int ITEM_TPB = 256;            // threads of the projection kernel
constexpr int MAX_BATCH_VARIATES = 8;

struct SetupChunk {
    int first, count;
    PageDev pg[SETUP_CHUNK];
};

// Copies the host-set fields of a chunk of pages into the device table
// (the device-set offsets are left alone).
__global__ void kb_setup(SetupChunk c, PageDev* __restrict__ pages)
{
    const int i = threadIdx.x;
    if (i >= c.count) return;
    PageDev& d = pages[c.first + i];
    const PageDev& h = c.pg[i];
    d.cube = h.cube;
    d.labels = h.labels;
    d.out = h.out;
    d.eigvals = h.eigvals;
    d.dm = h.dm;
    d.tiles = h.tiles;
    d.P = h.P;
    d.tile0 = h.tile0;
    d.item0 = h.item0;
    d.B = h.B;
    d.K = h.K;
    d.k = h.k;
    d.ntiles = h.ntiles;
    d.vec = h.vec;
    d.v8 = h.v8;
}

// Page of every label tile and every projection item (one CTA per page).
__global__ void kb_fill_pages(const PageDev* __restrict__ pages, int gpi, int* __restrict__ tile_page,
                              int* __restrict__ item_page)
{
    const int p = blockIdx.x;
    const PageDev& pg = pages[p];
    for (int t = threadIdx.x; t < pg.ntiles; t += blockDim.x) tile_page[pg.tile0 + t] = p;
    if (pg.v8) {
        const long long per = static_cast<long long>(gpi) * ITEM_TPB;
        const long long items = (pg.P / 8 + per - 1) / per;
        for (long long i = threadIdx.x; i < items; i += blockDim.x) item_page[pg.item0 + i] = p;
    }
}

struct Quad {
    unsigned long long v[4];
};

// Block-wide exclusive scan of four counters per thread (1024 threads).
__device__ Quad block_scan4(const Quad& x, Quad* warp_tot, Quad& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    Quad inc = x;
    #pragma unroll
    for (int q = 0; q < 4; ++q)
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, inc.v[q], o);
            if (lane >= o) inc.v[q] += u;
        }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    Quad before, all;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        unsigned long long b = 0, a = 0;
        for (int w = 0; w < nw; ++w) {
            const unsigned long long t = warp_tot[w].v[q];
            b += (w < warp) ? t : 0ull;
            a += t;
        }
        before.v[q] = b + inc.v[q] - x.v[q];
        all.v[q] = a;
    }
    __syncthreads();  // warp_tot is reused by the next chunk
    total = all;
    return before;
}

// One CTA of 1024 threads, one page per thread per chunk: training rows,
// pooled matrix words, moment units and range items of every page, their
// prefix sums over the pages, and the capacity check of the pool.
__global__ void __launch_bounds__(1024)
kb_pool_scan(PageDev* __restrict__ pages, int n, BatchTotals* __restrict__ tot, unsigned long long cap_rows,
             unsigned long long cap_xtr)
{
    __shared__ Quad warp_tot[32];
    unsigned long long run[4] = {0ull, 0ull, 0ull, 0ull};
    for (int base = 0; base < n; base += blockDim.x) {
        const int p = base + threadIdx.x;
        Quad x = {{0ull, 0ull, 0ull, 0ull}};
        if (p < n) {
            const PageDev& pg = pages[p];
            if (pg.dm->status == 0) {
                unsigned long long rows = 0, units = 0;
                for (int c = 0; c < pg.K; ++c) {
                    const unsigned long long nc = pg.dm->cls_count[c];
                    rows += nc;
                    units += (nc + 255) / 256;
                }
                x.v[0] = rows;
                x.v[1] = rows * static_cast<unsigned long long>(cva::xtr_row(pg.B));
                x.v[2] = units;
                x.v[3] = (rows + cva::BATCH_ROWS_PER_ITEM - 1) / cva::BATCH_ROWS_PER_ITEM;
            }
        }
        Quad total;
        const Quad ex = block_scan4(x, warp_tot, total);
        if (p < n) {
            PageDev& pg = pages[p];
            pg.row0 = run[0] + ex.v[0];
            pg.xoff = run[1] + ex.v[1];
            pg.unit0 = run[2] + ex.v[2];
            pg.titem0 = run[3] + ex.v[3];
            pg.nrows = x.v[0];
            if (x.v[0] && (pg.row0 + x.v[0] > cap_rows || pg.xoff + x.v[1] > cap_xtr))
                atomicCAS(&pg.dm->status, 0, CVA_ERR_CAPACITY);
        }
        #pragma unroll
        for (int q = 0; q < 4; ++q) run[q] += total.v[q];
    }
    if (threadIdx.x == 0) {
        tot->rows = run[0];
        tot->xtr = run[1];
        tot->units = run[2];
        tot->titems = run[3];
    }
}

__global__ void kb_status(const DevModel* __restrict__ dms, int n, int* __restrict__ status)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) {
        const DevModel* dm = dms + p;
        const int st = dm->status;
        status[p] = (st == 0 && !dm->fitted) ? CVA_ERR_NOT_FITTED : st;
    }
}

}  // namespace

struct cva_batch {
    int device;
    int num_sms;
    int max_pages;
    long long tiles_cap;   // words of the tile pool
    long long max_train;   // rows of the training pools
    DevModel* dms;
    PageDev* pages;
    unsigned int* tiles;
    unsigned int* list;
    uint16_t* xtr;
    BatchTotals* tot;
    int* status;
    int* tile_page;        // page of every label tile
    int* item_page;        // page of every projection item
    long long max_items;   // entries of item_page
    int gpi;               // pixel groups (TPB x 8 pixels) per projection item
    int grid_per_sm;       // persistent projection CTAs per SM, each on a contiguous run of items (0: one CTA per item)
    PageDev* host_pages;   // scratch for building the table
    // side streams and events: the projection launches of the variate counts
    // run side by side (fork from and join to the caller's stream; a
    // captured graph records them as parallel branches)
    cudaStream_t side[MAX_BATCH_VARIATES];
    cudaEvent_t fork;
    cudaEvent_t join[MAX_BATCH_VARIATES];
};

namespace {

void free_batch(cva_batch* b)
{
    cudaFree(b->dms);
    cudaFree(b->pages);
    cudaFree(b->tiles);
    cudaFree(b->list);
    cudaFree(b->xtr);
    cudaFree(b->tot);
    cudaFree(b->status);
    cudaFree(b->tile_page);
    cudaFree(b->item_page);
    for (int i = 0; i < MAX_BATCH_VARIATES; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete[] b->host_pages;
    delete b;
}

// Host-side page table and the batch's sizes; returns CVA_OK or an error.
// The table holds the pages sorted by their variate count k (stable), so that
// the projection items of each k form one range, projected by one launch of
// the kernel compiled for that k; page i keeps model block i.
struct Plan {
    long long tiles_total;
    long long items_total;
    long long kbeg[MAX_BATCH_VARIATES + 1], kend[MAX_BATCH_VARIATES + 1];  // items of each k
    int max_b, max_k;
};

int plan_batch(cva_batch* b, const cva_page* pages, int n, Plan* plan)
{
    if (!b || !pages || n < 1 || n > b->max_pages) return CVA_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const cva_page& q = pages[i];
        if (q.B < 1 || q.B > CVA_MAX_BANDS || q.K < 2 || q.K > CVA_MAX_CLASSES || q.H < 1 || q.W < 1 ||
            q.k < 1 || q.k > q.B || q.k > MAX_BATCH_VARIATES)
            return CVA_ERR_INVALID_ARG;
        if (static_cast<long long>(q.H) * q.W >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
        if (reinterpret_cast<uintptr_t>(q.cube) % 2 != 0) return CVA_ERR_INVALID_ARG;
        if (!device_visible(q.cube) || !device_visible(q.labels) || !device_visible(q.out) ||
            (q.eigvals && !device_visible(q.eigvals)))
            return CVA_ERR_INVALID_ARG;
    }
    long long tile0 = 0, item0 = 0, words = 0;
    int max_b = 1, max_k = 1;
    int t = 0;  // table position
    plan->kbeg[0] = plan->kend[0] = 0;
    for (int kk = 1; kk <= MAX_BATCH_VARIATES; ++kk) {
        plan->kbeg[kk] = item0;
        for (int i = 0; i < n; ++i) {
            const cva_page& q = pages[i];
            if (q.k != kk) continue;
            const long long P = static_cast<long long>(q.H) * q.W;
            const long long ntiles = (P + cva::LABEL_TILE - 1) / cva::LABEL_TILE;
            PageDev& d = b->host_pages[t++];
            std::memset(&d, 0, sizeof(d));
            d.cube = q.cube;
            d.labels = q.labels;
            d.out = q.out;
            d.eigvals = q.eigvals;
            d.dm = b->dms + i;
            d.tiles = b->tiles + words;
            d.P = P;
            d.tile0 = tile0;
            d.B = q.B;
            d.K = q.K;
            d.k = q.k;
            d.ntiles = static_cast<int>(ntiles);
            d.vec = (reinterpret_cast<uintptr_t>(q.labels) % 16 == 0) ? 1 : 0;
            d.v8 = (P % 8 == 0) && (reinterpret_cast<uintptr_t>(q.cube) % 16 == 0) &&
                   (reinterpret_cast<uintptr_t>(q.out) % 8 == 0);
            d.item0 = item0;
            if (d.v8) {
                const long long groups = P / 8;
                const long long per = static_cast<long long>(b->gpi) * ITEM_TPB;
                item0 += (groups + per - 1) / per;
            }
            words += ntiles * (q.K + 1);
            tile0 += ntiles;
            if (q.B > max_b) max_b = q.B;
            if (q.k > max_k) max_k = q.k;
        }
        plan->kend[kk] = item0;
    }
    if (words > b->tiles_cap || tile0 > b->tiles_cap || item0 > b->max_items) return CVA_ERR_CAPACITY;
    if (tile0 >= (1LL << 31)) return CVA_ERR_INVALID_ARG;
    plan->tiles_total = tile0;
    plan->items_total = item0;
    plan->max_b = max_b;
    plan->max_k = max_k;
    return CVA_OK;
}

cudaError_t upload_pages(cva_batch* b, int n, cudaStream_t s)
{
    for (int first = 0; first < n; first += SETUP_CHUNK) {
        SetupChunk c;
        std::memset(&c, 0, sizeof(c));
        c.first = first;
        c.count = (n - first) < SETUP_CHUNK ? (n - first) : SETUP_CHUNK;
        std::memcpy(c.pg, b->host_pages + first, sizeof(PageDev) * c.count);
        kb_setup<<<1, SETUP_CHUNK, 0, s>>>(c, b->pages);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    kb_fill_pages<<<n, 256, 0, s>>>(b->pages, b->gpi, b->tile_page, b->item_page);
    return cudaGetLastError();
}

int projection_grid(const cva_batch* b, long long items)
{
    if (b->grid_per_sm <= 0) return static_cast<int>(items < (1LL << 30) ? items : (1LL << 30));
    return b->num_sms * b->grid_per_sm;
}

cudaError_t launch_projection(cva_batch* b, int n, const Plan& plan, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (int k = 1; k <= MAX_BATCH_VARIATES && e == cudaSuccess; ++k) {
        const long long items = plan.kend[k] - plan.kbeg[k];
        if (items <= 0) continue;
        cudaStream_t t = b->side[k - 1];
        e = cudaStreamWaitEvent(t, b->fork, 0);
        if (e == cudaSuccess)
            e = cva::launch_batch_project(b->pages, b->item_page, plan.kbeg[k], plan.kend[k], b->gpi,
                                          projection_grid(b, items), k, t);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[k - 1], t);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[k - 1], 0);
    }
    // pages the batched kernel does not take (pixel count or alignment)
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const PageDev& d = b->host_pages[i];
        if (d.v8) continue;
        e = cva::launch_project(d.cube, d.B, d.P, d.dm, d.k, nullptr, d.out, d.dm->train_range, nullptr,
                                b->num_sms, s);
    }
    return e;
}

cudaError_t run_batch(cva_batch* b, int n, const Plan& plan, cudaStream_t s, bool project = true)
{
    cudaError_t e = upload_pages(b, n, s);
    if (e == cudaSuccess) e = cva::launch_batch_tile_count(b->pages, b->tile_page, plan.tiles_total, s);
    if (e == cudaSuccess) {
        kb_pool_scan<<<1, 1024, 0, s>>>(b->pages, n, b->tot, static_cast<unsigned long long>(b->max_train),
                                        static_cast<unsigned long long>(b->max_train) * XTR_POOL_ROW);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cva::launch_batch_tile_compact(b->pages, b->tile_page, plan.tiles_total, b->list, s);
    if (e == cudaSuccess)
        e = cva::launch_batch_gather_moments(b->pages, n, b->tot, b->list, b->xtr, plan.max_b, b->num_sms, s);
    if (e == cudaSuccess) e = cva::launch_batch_finalize(b->pages, n, s);
    if (e == cudaSuccess)
        e = cva::launch_batch_train_range(b->pages, n, b->tot, b->xtr, plan.max_k, b->num_sms, s);
    if (e == cudaSuccess && project) e = launch_projection(b, n, plan, s);
    return e;
}

}  // namespace

extern "C" {

int cva_batch_create(int max_pages, int64_t max_pixels, int64_t max_train, cva_batch** out)
{
    if (!out) return CVA_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_pages < 1 || max_pages > CVA_MAX_BATCH_PAGES || max_pixels < 1 || max_train < 1 ||
        max_train >= (1LL << 32))
        return CVA_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CVA_ERR_CUDA;
    cva_batch* b = new (std::nothrow) cva_batch;
    if (!b) return CVA_ERR_INVALID_ARG;
    std::memset(b, 0, sizeof(*b));
    b->device = dev;
    b->num_sms = sms;
    b->max_pages = max_pages;
    b->tiles_cap = (max_pixels / cva::LABEL_TILE + max_pages) * static_cast<long long>(CVA_MAX_CLASSES + 1);
    b->max_items = max_pixels / (8 * ITEM_TPB) + max_pages;
    b->max_train = max_train;
    b->gpi = 2;
    b->grid_per_sm = 2;
    b->host_pages = new (std::nothrow) PageDev[max_pages];
    bool ok = b->host_pages != nullptr;
    ok = ok && cudaMalloc(&b->dms, sizeof(DevModel) * max_pages) == cudaSuccess;
    ok = ok && cudaMalloc(&b->pages, sizeof(PageDev) * max_pages) == cudaSuccess;
    ok = ok && cudaMalloc(&b->tiles, sizeof(unsigned int) * b->tiles_cap) == cudaSuccess;
    ok = ok && cudaMalloc(&b->list, sizeof(unsigned int) * max_train) == cudaSuccess;
    ok = ok && cudaMalloc(&b->xtr, sizeof(uint16_t) * max_train * XTR_POOL_ROW) == cudaSuccess;
    ok = ok && cudaMalloc(&b->tot, sizeof(BatchTotals)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->status, sizeof(int) * max_pages) == cudaSuccess;
    ok = ok && cudaMalloc(&b->tile_page, sizeof(int) * b->tiles_cap) == cudaSuccess;
    ok = ok && cudaMalloc(&b->item_page, sizeof(int) * b->max_items) == cudaSuccess;
    ok = ok && cudaMemset(b->dms, 0, sizeof(DevModel) * max_pages) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < MAX_BATCH_VARIATES && ok; ++i) {
        ok = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaMemset(b->pages, 0, sizeof(PageDev) * max_pages) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return CVA_ERR_CUDA;
    }
    *out = b;
    return CVA_OK;
}

void cva_batch_destroy(cva_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    free_batch(b);
}

int cva_fit_project_batched(cva_batch* b, const cva_page* pages, int n, void* stream)
{
    Plan plan;
    const int rc = plan_batch(b, pages, n, &plan);
    if (rc != CVA_OK) return rc;
    return run_batch(b, n, plan, static_cast<cudaStream_t>(stream)) == cudaSuccess ? CVA_OK : CVA_ERR_CUDA;
}

int cva_fit_batched(cva_batch* b, const cva_page* pages, int n, void* stream)
{
    Plan plan;
    const int rc = plan_batch(b, pages, n, &plan);
    if (rc != CVA_OK) return rc;
    return run_batch(b, n, plan, static_cast<cudaStream_t>(stream), false) == cudaSuccess ? CVA_OK : CVA_ERR_CUDA;
}

int cva_project_batched(cva_batch* b, const cva_page* pages, int n, void* stream)
{
    Plan plan;
    const int rc = plan_batch(b, pages, n, &plan);
    if (rc != CVA_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = upload_pages(b, n, s);
    if (e == cudaSuccess) e = launch_projection(b, n, plan, s);
    return e == cudaSuccess ? CVA_OK : CVA_ERR_CUDA;
}

int cva_batch_status(cva_batch* b, int n, int* status, void* stream)
{
    if (!b || !status || n < 1 || n > b->max_pages) return CVA_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    kb_status<<<(n + 255) / 256, 256, 0, s>>>(b->dms, n, b->status);
    if (cudaGetLastError() != cudaSuccess) return CVA_ERR_CUDA;
    if (cudaMemcpyAsync(status, b->status, sizeof(int) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CVA_ERR_CUDA;
    for (int i = 0; i < n; ++i)
        if (status[i] != CVA_OK) return status[i];
    return CVA_OK;
}

int cva_batch_tune(cva_batch* b, const cva_page* pages, int n, void* stream, int* chosen)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan plan;
    int rc = plan_batch(b, pages, n, &plan);
    if (rc != CVA_OK) return rc;
    if (run_batch(b, n, plan, s) != cudaSuccess) return CVA_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return CVA_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return CVA_ERR_CUDA;
    }
    // the candidates stated in cva.h: 1, 2, 4, 8, 16 or 32 groups a work item
    static const int kGpi[] = {1, 2, 4, 8, 16, 32};
    static const int kGrid[] = {2, 0};
    constexpr int NGPI = static_cast<int>(sizeof(kGpi) / sizeof(kGpi[0]));
    float best = 0.0f;
    int best_gpi = b->gpi, best_grid = b->grid_per_sm;
    bool fail = false;
    for (int gi = 0; gi < 2 && !fail; ++gi)
        for (int pi = 0; pi < NGPI && !fail; ++pi) {
            b->gpi = kGpi[pi];
            b->grid_per_sm = kGrid[gi];
            if (plan_batch(b, pages, n, &plan) != CVA_OK || upload_pages(b, n, s) != cudaSuccess) {
                fail = true;
                break;
            }
            for (int w = 0; w < 2 && !fail; ++w) fail = launch_projection(b, n, plan, s) != cudaSuccess;
            fail = fail || cudaEventRecord(e0, s) != cudaSuccess;
            for (int r = 0; r < 5 && !fail; ++r) fail = launch_projection(b, n, plan, s) != cudaSuccess;
            fail = fail || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess;
            float ms = 0.0f;
            fail = fail || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
            if (!fail && (best == 0.0f || ms < best)) {
                best = ms;
                best_gpi = b->gpi;
                best_grid = b->grid_per_sm;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->gpi = best_gpi;
    b->grid_per_sm = best_grid;
    if (fail) return CVA_ERR_CUDA;
    if (chosen) {
        chosen[0] = b->gpi;
        chosen[1] = b->grid_per_sm;
    }
    return CVA_OK;
}

}  // extern "C"
