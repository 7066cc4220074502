// ggns_noalloc.cu -- allocation-free variant of the k-NN component finder.
//
// Some callers cannot allocate device memory at the time they need the
// clustering step: a host framework that owns every device allocation through
// its own pool, or a process whose device-memory budget is fixed once at start
// time.  ns_knn_components_noalloc serves them: its scratch (labels, cluster
// sizes, neighbour ranks, last neighbour keys, component count) is one
// file-scope __device__ array, so a call allocates and frees nothing.
#include <mutex>

#include "ggns_iter.cuh"

namespace {

using ggns::CMAX;
using ggns::KNN_K;

constexpr int NOALLOC_MAX_POINTS = 4096;

struct KnnScratch {
    int label[NOALLOC_MAX_POINTS];
    int csize[CMAX];
    int ncomp;
    int pad_[63];  // keeps lastkey on a 256-byte boundary
    unsigned long long lastkey[NOALLOC_MAX_POINTS];
    int nbr[NOALLOC_MAX_POINTS * KNN_K];
};
static_assert((offsetof(KnnScratch, lastkey) % 256) == 0, "lastkey alignment");

// Resident on every device that loads the library, until the process exits
// (about 304 KiB).  Shared by every call on that device.
static __device__ __align__(256) KnnScratch g_knn_scratch;

// One cluster holding all m points: label 0, size m.
__global__ void k_noalloc_reset(KnnScratch *s, int m)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) s->label[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x < CMAX) s->csize[threadIdx.x] = (threadIdx.x == 0) ? m : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) s->ncomp = 0;
}

constexpr int MAX_DEVICES = 256;
std::mutex g_mu;
KnnScratch *g_dev_ptr[MAX_DEVICES] = {};
void *g_dev_ctx[MAX_DEVICES] = {};  // the context the address was looked up in

// The current driver context, through the runtime's driver entry point (no link to
// libcuda); nullptr if it cannot be queried.  A device reset or a new primary
// context reloads the module and moves the array, so the cached address is kept
// per context, not per device.
void *current_context()
{
    using GetCtx = int (*)(void **);
    static GetCtx fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetCtx>(f);
    }();
    void *c = nullptr;
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

}  // namespace

extern "C" ns_status ns_knn_components_noalloc(const float *x_dev, int m, int d, int *comp_dev, int *n_comp_host,
                                               void *stream)
{
    if (m < 1 || m > NOALLOC_MAX_POINTS) {
        ggns::set_global_error("ns_knn_components_noalloc: m must be in [1, 4096] (the size of its static scratch)");
        return NS_ERR_ARG;
    }
    if (d < 1 || d > ggns::DMAX || !x_dev || !comp_dev || !n_comp_host) {
        ggns::set_global_error("ns_knn_components_noalloc: need 1 <= d <= 512 and non-NULL pointers");
        return NS_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        ggns::set_global_error("ns_knn_components_noalloc: no current CUDA device");
        return NS_ERR_CUDA;
    }
    KnnScratch *p;
    {
        // set-up, once per device with that device current: the device address of
        // the scratch (the host-side name is only a stand-in for it)
        std::lock_guard<std::mutex> lk(g_mu);
        void *cur = current_context();
        if (!g_dev_ptr[dev] || !cur || cur != g_dev_ctx[dev]) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_knn_scratch);
            if (e != cudaSuccess) {
                ggns::set_global_error(cudaGetErrorString(e));
                return NS_ERR_CUDA;
            }
            g_dev_ptr[dev] = static_cast<KnnScratch *>(addr);
            g_dev_ctx[dev] = current_context();
        }
        p = g_dev_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_noalloc_reset<<<(m + 255) / 256, 256, 0, s>>>(p, m);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = ggns::launch_knn_components(x_dev, m, d, p->label, p->csize, p->nbr, comp_dev, p->lastkey, &p->ncomp, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, &p->ncomp, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        ggns::set_global_error(cudaGetErrorString(e));
        return NS_ERR_CUDA;
    }
    *n_comp_host = h;
    return NS_OK;
}
