// ggns_kind_impl.cuh -- instantiates the walker-layout kernels of one likelihood
// kind (GGNS_KIND) for every walker tile and exposes them through a KindLaunch.
#pragma once

#include "ggns_iter.cuh"
#include "ggns_kernels.cuh"

namespace ggns {
namespace GGNS_KIND_NS {

constexpr int KIND = GGNS_KIND;

template <int G, int E>
static cudaError_t prior_t(const DevCtx &C, const int *runs, int nr, int max_n, size_t smem, int pis, cudaStream_t s)
{
    const int gpc = HSS_THREADS / G;
    int bx = (max_n + gpc - 1) / gpc;
    if (bx > 1024) bx = 1024;
    k_prior_init<KIND, G, E><<<dim3(bx, nr), HSS_THREADS, smem, s>>>(C, runs, pis);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t hss_t(const DevCtx &C, const int *runs, int nr, int max_k, int phase, size_t smem, int pis,
                         cudaStream_t s)
{
    const int gpc = HSS_THREADS / G;
    const int bx = (max_k + gpc - 1) / gpc;
    k_hss<KIND, G, E><<<dim3(bx, nr), HSS_THREADS, smem, s>>>(C, runs, phase, pis);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t lik_t(const DevCtx &C, int run, const float *x, long n, int mode, float *logl, float *grad,
                         const float *gout, float *gmu, size_t smem, int pis, cudaStream_t s)
{
    const int gpc = HSS_THREADS / G;
    long bx = (n + gpc - 1) / gpc;
    if (bx > 65535) bx = 65535;
    if (bx < 1) bx = 1;
    k_lik_points<KIND, G, E><<<(unsigned)bx, HSS_THREADS, smem, s>>>(C, run, x, n, mode, logl, grad, gout, gmu, pis);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t grad_t(const DevCtx &C, int run, double logz, double *part, int nb, size_t smem, int pis,
                          cudaStream_t s)
{
    k_grad_means<KIND, G, E><<<nb, HSS_THREADS, smem, s>>>(C, run, logz, part, pis);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t hss1_t(const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R, const long *rec_base,
                          size_t smem, int pis, cudaStream_t s)
{
    const int gpc = HSS_THREADS / G;
    const int bx = (max_k + gpc - 1) / gpc;
    k_hss1<KIND, G, E><<<dim3(bx, nr), HSS_THREADS, smem, s>>>(C, runs, R, rec_base, pis, 0);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t eval_new_t(const DevCtx &C, const int *runs, int nr, int max_k, size_t smem, int pis, cudaStream_t s)
{
    const int gpc = HSS_THREADS / G;
    const int bx = (max_k + gpc - 1) / gpc;
    k_eval_new<KIND, G, E><<<dim3(bx, nr), HSS_THREADS, smem, s>>>(C, runs, pis);
    return cudaGetLastError();
}
template <int G, int E>
static cudaError_t occ_t(size_t smem, int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_hss1<KIND, G, E>, HSS_THREADS, smem);
}
template <int G, int E>
static cudaError_t smem_t(size_t smem)
{
    if (smem <= 48 * 1024) return cudaSuccess;
    const int v = (int)smem;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute((const void *)k_prior_init<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute((const void *)k_hss<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute((const void *)k_hss1<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute((const void *)k_lik_points<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute((const void *)k_eval_new<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_grad_means<KIND, G, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, v);
}

#define GGNS_DISPATCH(FN, ...)                                   \
    switch (tile) {                                              \
    case 0: return FN<1, 2>(__VA_ARGS__);                        \
    case 1: return FN<1, 4>(__VA_ARGS__);                        \
    case 2: return FN<2, 4>(__VA_ARGS__);                        \
    case 3: return FN<4, 4>(__VA_ARGS__);                        \
    case 4: return FN<8, 4>(__VA_ARGS__);                        \
    case 5: return FN<16, 4>(__VA_ARGS__);                       \
    case 6: return FN<32, 4>(__VA_ARGS__);                       \
    case 7: return FN<32, 8>(__VA_ARGS__);                       \
    case 8: return FN<32, 16>(__VA_ARGS__);                      \
    case 9: return FN<4, 8>(__VA_ARGS__);                        \
    case 10: return FN<16, 2>(__VA_ARGS__);                      \
    case 11: return FN<8, 8>(__VA_ARGS__);                       \
    case 12: return FN<16, 8>(__VA_ARGS__);                      \
    case 13: return FN<32, 1>(__VA_ARGS__);                      \
    case 14: return FN<32, 2>(__VA_ARGS__);                      \
    default: return cudaErrorInvalidValue;                       \
    }

static cudaError_t prior(int tile, const DevCtx &C, const int *runs, int nr, int max_n, size_t smem, int pis,
                         cudaStream_t s)
{
    GGNS_DISPATCH(prior_t, C, runs, nr, max_n, smem, pis, s)
}
static cudaError_t hss(int tile, const DevCtx &C, const int *runs, int nr, int max_k, int phase, size_t smem, int pis,
                       cudaStream_t s)
{
    GGNS_DISPATCH(hss_t, C, runs, nr, max_k, phase, smem, pis, s)
}
static cudaError_t lik(int tile, const DevCtx &C, int run, const float *x, long n, int mode, float *logl, float *grad,
                       const float *gout, float *gmu, size_t smem, int pis, cudaStream_t s)
{
    GGNS_DISPATCH(lik_t, C, run, x, n, mode, logl, grad, gout, gmu, smem, pis, s)
}
static cudaError_t grad(int tile, const DevCtx &C, int run, double logz, double *part, int nb, size_t smem, int pis,
                        cudaStream_t s)
{
    GGNS_DISPATCH(grad_t, C, run, logz, part, nb, smem, pis, s)
}
static cudaError_t smem_attr(int tile, size_t smem)
{
    GGNS_DISPATCH(smem_t, smem)
}
static cudaError_t hss1(int tile, const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R,
                        const long *rec_base, size_t smem, int pis, cudaStream_t s)
{
    GGNS_DISPATCH(hss1_t, C, runs, nr, max_k, R, rec_base, smem, pis, s)
}
static cudaError_t hss1_occ(int tile, size_t smem, int *blocks_per_sm)
{
    GGNS_DISPATCH(occ_t, smem, blocks_per_sm)
}
static cudaError_t eval_new(int tile, const DevCtx &C, const int *runs, int nr, int max_k, size_t smem, int pis,
                            cudaStream_t s)
{
    GGNS_DISPATCH(eval_new_t, C, runs, nr, max_k, smem, pis, s)
}

// The CTA-cooperative single pass (dense kinds, one walker per warp): tiles 6, 7, 8.
template <int E>
static cudaError_t coop_t(const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R, const long *rec_base,
                          size_t smem, int tr, cudaStream_t s)
{
    const int wpc = COOP_THREADS / 32;
    const int bx = (max_k + wpc - 1) / wpc;
    k_hss1<KIND, 32, E, true><<<dim3(bx, nr), COOP_THREADS, smem, s>>>(C, runs, R, rec_base, 0, tr);
    return cudaGetLastError();
}
template <int E>
static cudaError_t coop_occ_t(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k_hss1<KIND, 32, E, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_hss1<KIND, 32, E, true>, COOP_THREADS, smem);
}
// The same CTA form with the contraction on the tensor cores (tr = 1).
template <int E>
static cudaError_t tc_t(const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R, const long *rec_base,
                        size_t smem, cudaStream_t s)
{
    const int wpc = COOP_THREADS / 32;
    const int bx = (max_k + wpc - 1) / wpc;
    k_hss1<KIND, 32, E, true, true><<<dim3(bx, nr), COOP_THREADS, smem, s>>>(C, runs, R, rec_base, 0, 0);
    return cudaGetLastError();
}
template <int E>
static cudaError_t tc_occ_t(size_t smem, int *blocks_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k_hss1<KIND, 32, E, true, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_hss1<KIND, 32, E, true, true>, COOP_THREADS,
                                                         smem);
}
template <int KD>
static cudaError_t coop_dispatch(int tile, bool occ, bool tcore, const DevCtx *C, const int *runs, int nr, int max_k,
                                 const RecView *R, const long *rec_base, size_t smem, int tr, int *blocks_per_sm,
                                 cudaStream_t s)
{
    if constexpr (KD == NS_LIK_DENSE_GAUSS || KD == NS_LIK_DENSE_MIX) {
        if (tcore) {
            switch (tile) {
            case 6: return occ ? tc_occ_t<4>(smem, blocks_per_sm) : tc_t<4>(*C, runs, nr, max_k, *R, rec_base, smem, s);
            case 7: return occ ? tc_occ_t<8>(smem, blocks_per_sm) : tc_t<8>(*C, runs, nr, max_k, *R, rec_base, smem, s);
            case 8: return occ ? tc_occ_t<16>(smem, blocks_per_sm) : tc_t<16>(*C, runs, nr, max_k, *R, rec_base, smem, s);
            default: return cudaErrorInvalidValue;
            }
        }
        switch (tile) {
        case 6: return occ ? coop_occ_t<4>(smem, blocks_per_sm) : coop_t<4>(*C, runs, nr, max_k, *R, rec_base, smem, tr, s);
        case 7: return occ ? coop_occ_t<8>(smem, blocks_per_sm) : coop_t<8>(*C, runs, nr, max_k, *R, rec_base, smem, tr, s);
        case 8: return occ ? coop_occ_t<16>(smem, blocks_per_sm) : coop_t<16>(*C, runs, nr, max_k, *R, rec_base, smem, tr, s);
        default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorInvalidValue;
    }
}
static cudaError_t hss1_coop(int tile, const DevCtx &C, const int *runs, int nr, int max_k, const RecView &R,
                             const long *rec_base, size_t smem, int tr, cudaStream_t s)
{
    return coop_dispatch<KIND>(tile, false, tr == 0, &C, runs, nr, max_k, &R, rec_base, smem, tr, nullptr, s);
}
static cudaError_t hss1_coop_occ(int tile, size_t smem, int tr, int *blocks_per_sm)
{
    return coop_dispatch<KIND>(tile, true, tr == 0, nullptr, nullptr, 0, 0, nullptr, nullptr, smem, tr, blocks_per_sm,
                               nullptr);
}

}  // namespace GGNS_KIND_NS
}  // namespace ggns
